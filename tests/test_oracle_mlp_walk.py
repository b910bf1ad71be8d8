"""Pins of the oracle's learned-criterion walk, its evaluation on given lists and
the three features that the hand-built geometry of test_oracle_mlp.py leaves
out. Each check ties an oracle function to something fixed outside it:

* ``forces_on_lists`` on the oracle's own key-ordered lists equals
  ``forces`` bit for bit, and on the theta = 0 lists equals the direct sum O1;
* the learned walk reduces to plain theta walks (themselves pinned to the
  direct sum and to hand-derived lists) in every limit where the rule says it
  must: an empty band, tau = +inf / -inf, a constant network at and just
  above tau, every input out of range;
* point cells (h = 0) inside the band are accepted: with theta_lo = 0 and
  a network that opens everything, the forces equal the direct sum and the
  cell-list lengths equal a brute-force count;
* coincident particles at eps = 0 give finite results equal to O1's;
* features 2, 5 and 11 on a geometry whose values are worked out by hand.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.mlp as M
from paper_1005_5384_gb300 import workloads as W


def _plummer(n, seed):
    pos, m = W.plummer(n, seed=seed)
    return pos, m


@pytest.fixture(scope="module")
def tree():
    pos, m = _plummer(3000, 21)
    return O.Tree(pos, m, n_leaf=8, n_group=16)


def _open_net(seed=4):
    """A random network whose inputs are never out of range."""
    return dict(w=M.init(seed), mu=np.zeros(12), sigma=np.ones(12), fmin=np.full(12, -np.inf),
                fmax=np.full(12, np.inf))


def _same(a, b):
    """Bitwise equality of two oracle results (acc, pot, n_pp, n_pc)."""
    for x, y in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(x, y)


# ---------------------------------------------------------------- O6 on given lists

def test_forces_on_lists_equals_tree_forces_bitwise(tree):
    """The oracle sums the cell list, then the leaf list, each in key order; the
    same lists handed to forces_on_lists in key order give the same bits."""
    T = tree
    eps, theta = 0.01, 0.6
    groups = W.sample_indices(T.n_groups, 40, seed=3)
    acc, pot, _, _, _ = T.forces(eps, theta, groups=groups, nthreads=2)
    for g in groups:
        cells, leaves = T.lists(int(g), theta)
        cells = cells[np.argsort(T.key[cells], kind="stable")]
        leaves = leaves[np.argsort(T.key[leaves], kind="stable")]
        a, p = T.forces_on_lists(int(g), cells, leaves, eps)
        mem = T.cell_members(int(T.groups[g]))
        np.testing.assert_array_equal(a, acc[mem])
        np.testing.assert_array_equal(p, pot[mem])


def test_forces_on_lists_at_theta_zero_is_direct_sum(tree):
    """theta = 0 opens everything: the leaf lists cover all particles and the
    evaluation on them is the direct sum O1 (pinned by closed forms)."""
    T = tree
    eps = 0.02
    groups = W.sample_indices(T.n_groups, 12, seed=5)
    for g in groups:
        cells, leaves = T.lists(int(g), 0.0)
        assert len(cells) == 0
        mem = T.cell_members(int(T.groups[g]))
        a, p = T.forces_on_lists(int(g), cells, leaves, eps, G=1.3)
        ad, pd = O.direct(T.pos, T.mass, eps, G=1.3, targets=mem, nthreads=1)
        np.testing.assert_allclose(a, ad, rtol=1e-12, atol=1e-12 * np.abs(ad).max())
        np.testing.assert_allclose(p, pd, rtol=1e-12)


def test_forces_on_lists_changes_with_a_dropped_entry(tree):
    """A list with one accepted cell left out gives a different result (the
    function reads every entry it is given)."""
    T = tree
    g = int(W.sample_indices(T.n_groups, 1, seed=8)[0])
    cells, leaves = T.lists(g, 0.6)
    assert len(cells) > 2
    a, _ = T.forces_on_lists(g, cells, leaves, 0.01)
    b, _ = T.forces_on_lists(g, cells[1:], leaves, 0.01)
    assert np.abs(a - b).max() > 0


# ---------------------------------------------------------------- O8 walk limits

def test_empty_band_is_the_theta_walk(tree):
    """theta_lo = theta_hi = theta: every child is decided by the band, the
    network is never consulted and the walk is the plain theta walk."""
    T = tree
    net = _open_net()
    for theta in (0.4, 0.7):
        ref = T.forces(0.01, theta, nthreads=2)
        got = T.forces_mlp(0.01, net, 0.0, theta, theta, 99.0, nthreads=2)
        _same(got, ref)
        assert got[4] == 0


@pytest.mark.parametrize("tau,walk", [(math.inf, "hi"), (-math.inf, "lo")])
def test_tau_limits_give_the_band_walks(tree, tau, walk):
    """A network that accepts everything leaves only what the theta_hi test
    opens; one that opens everything leaves only what theta_lo accepts."""
    T = tree
    lo, hi = 0.45, 0.9
    got = T.forces_mlp(0.01, _open_net(), tau, lo, hi, 99.0, nthreads=2)
    ref = T.forces(0.01, hi if walk == "hi" else lo, nthreads=2)
    _same(got, ref)
    assert got[4] > 1000  # the network was consulted


def test_constant_network_threshold_is_strict(tree):
    """A network that predicts a constant c accepts iff c < tau: at tau = c it
    opens every band pair (theta_lo walk), just above c it accepts them all
    (theta_hi walk)."""
    T = tree
    p = {k: np.zeros(s) for k, s in M.SIZES}
    c = -3.0
    p["b3"][0] = c
    net = dict(w=M.pack(p), mu=np.zeros(12), sigma=np.ones(12), fmin=np.full(12, -np.inf),
               fmax=np.full(12, np.inf))
    lo, hi = 0.45, 0.9
    _same(T.forces_mlp(0.01, net, c, lo, hi, 99.0, nthreads=2), T.forces(0.01, lo, nthreads=2))
    _same(T.forces_mlp(0.01, net, math.nextafter(c, 0.0), lo, hi, 99.0, nthreads=2),
          T.forces(0.01, hi, nthreads=2))


def test_out_of_range_inputs_fall_back_to_theta_fb(tree):
    """With no input inside the training range every band pair is decided by the
    theta_fb test; for theta_lo <= theta_fb <= theta_hi that is the theta_fb
    walk exactly (the test is monotone in theta)."""
    T = tree
    net = _open_net()
    net["fmin"] = np.full(12, np.inf)
    got = T.forces_mlp(0.01, net, 0.0, 0.45, 0.9, 0.6, nthreads=2)
    _same(got, T.forces(0.01, 0.6, nthreads=2))
    assert got[4] == 0
    # one input out of range is enough
    net = _open_net()
    net["fmax"][7] = -np.inf
    got = T.forces_mlp(0.01, net, 0.0, 0.45, 0.9, 0.6, nthreads=2)
    _same(got, T.forces(0.01, 0.6, nthreads=2))


def test_point_cells_in_the_band_are_accepted():
    """theta_lo = 0 puts every cell that theta_hi does not open into the band;
    a network that opens everything then leaves exactly the point cells (single
    particles, h = 0) apart from the group accepted as exact monopoles: the
    forces equal the direct sum, and each group's cell list is the set of
    single-particle leaves whose position lies outside its box."""
    pos, m = _plummer(1200, 33)
    T = O.Tree(pos, m, n_leaf=2, n_group=8)
    eps = 0.01
    acc, pot, npp, npc, nm = T.forces_mlp(eps, _open_net(), -math.inf, 0.0, 0.5, 99.0, nthreads=2)
    ad, pd = O.direct(pos, m, eps, nthreads=2)
    np.testing.assert_allclose(acc, ad, rtol=1e-10, atol=1e-12 * np.abs(ad).max())
    np.testing.assert_allclose(pot, pd, rtol=1e-11)
    points = [c for c in range(T.n_cells) if T.leaf[c] and T.count[c] == 1]
    assert len(points) > 100
    f32 = np.float32
    for g in W.sample_indices(T.n_groups, 30, seed=2):
        gc = int(T.groups[g])
        outside = sum(1 for c in points
                      if not O.open_f32(T.bmin[gc].astype(f32), T.bmax[gc].astype(f32),
                                        T.cube[c, :3].astype(f32), 0.0, 0.5))
        mem = T.cell_members(gc)
        assert np.all(npc[mem] == outside), (g, npc[mem][0], outside)
    assert npc.sum() > 0 and nm > 0


# ---------------------------------------------------------------- coincident particles at eps = 0

def test_coincident_particles_at_zero_softening():
    """Two particles at one point, eps = 0: O1 leaves the pair out (zero force,
    finite potential from the rest); the tree walk, the learned walk and the
    evaluation on lists do the same and stay finite."""
    rng = np.random.default_rng(17)
    pos = rng.random((300, 3))
    pos[7] = pos[123]
    m = rng.random(300) + 0.5
    T = O.Tree(pos, m, n_leaf=4, n_group=8)
    ad, pd = O.direct(pos, m, 0.0, nthreads=1)
    assert np.all(np.isfinite(ad)) and np.all(np.isfinite(pd))
    ref = T.forces(0.0, 0.0, nthreads=1)
    np.testing.assert_allclose(ref[0], ad, rtol=1e-11, atol=1e-11 * np.abs(ad).max())
    got = T.forces_mlp(0.0, _open_net(), 0.0, 0.0, 0.0, 99.0, nthreads=1)
    _same(got, ref)
    g = int(T.group_of_particle()[7])
    cells, leaves = T.lists(g, 0.0)
    a, p = T.forces_on_lists(g, cells, leaves, 0.0)
    mem = T.cell_members(int(T.groups[g]))
    np.testing.assert_allclose(a, ad[mem], rtol=1e-11, atol=1e-11 * np.abs(ad).max())
    np.testing.assert_allclose(p, pd[mem], rtol=1e-12)
    aref = np.ones((300, 3))
    _, lab, _ = T.mlp_samples([g], 0.3, 0.0, aref)
    assert len(lab) > 0 and np.all(np.isfinite(lab))


# ---------------------------------------------------------------- features 2, 5, 11

def test_features_2_5_11_on_hand_worked_geometry():
    """Group a: four unit masses, box [0.5, 0.6]^3. Cell b: four particles of
    mass 2 at c +- (u, u, 0) and c +- (0, v, v) around c = (10.1, 10.1, 10.1),
    u = 0.1, v = 0.05. By hand:
      centre of mass of b = c; box of b = c +- (0.1, 0.1, 0.05): h = 0.1, l = 0.2,
      S = 4 * [[u^2, u^2, 0], [u^2, u^2 + v^2, v^2], [0, v^2, v^2]]
        = [[0.04, 0.04, 0], [0.04, 0.05, 0.01], [0, 0.01, 0.01]],
      |S|_F^2 = 0.04^2 + 0.05^2 + 0.01^2 + 2 (0.04^2 + 0 + 0.01^2)
              = 0.0042 + 2 * 0.0017 = 0.0076,
      feature 5 = sqrt(0.0076) / (8 * 0.2^2) = sqrt(0.0076) / 0.32 (without the
      doubled off-diagonal terms it would be sqrt(0.0042) / 0.32);
      C_a = centre of a's cube = (0.55, 0.55, 0.55): feature 2 = log2(9.55 sqrt 3);
      root centre of mass = (4 * 0.5625 + 8 * 10.1) / 12 per axis (a's mean
      coordinates are 0.5625 on x, y and z): feature 11 = log2(|C_a - com| sqrt 3)."""
    a = np.array([[0.5, 0.5, 0.5], [0.6, 0.5, 0.5], [0.5, 0.6, 0.5], [0.6, 0.6, 0.6]])
    # a's coordinates: x {0.5, 0.6, 0.5, 0.6}, y {0.5, 0.5, 0.6, 0.6}, z {0.5, 0.5, 0.5, 0.6}
    c = np.array([10.1, 10.1, 10.1])
    u, v = 0.1, 0.05
    b = np.array([c + [u, u, 0], c - [u, u, 0], c + [0, v, v], c - [0, v, v]])
    pos = np.vstack([a, b])
    m = np.array([1.0, 1, 1, 1, 2, 2, 2, 2])
    T = O.Tree(pos, m, n_leaf=4, n_group=4)
    ga = [g for g, cc in enumerate(T.groups) if T.count[cc] == 4 and T.bmax[cc, 0] < 1][0]
    cb = [k for k in range(T.n_cells) if T.count[k] == 4 and T.bmin[k, 0] > 9][0]
    f = T.mlp_features(ga, cb)
    assert f[5] == pytest.approx(math.sqrt(0.0076) / 0.32, rel=1e-12)
    assert f[2] == pytest.approx(math.log2(9.55 * math.sqrt(3.0)), rel=1e-12)
    mean_a = np.array([0.55, 0.55, 0.525])
    com_root = (4 * mean_a + 8 * c) / 12
    d11 = np.linalg.norm(np.array([0.55, 0.55, 0.55]) - com_root)
    assert f[11] == pytest.approx(math.log2(d11), rel=1e-12)
    # a cell with S = 0 (a single particle far away) has feature 5 = 0 and l = 0
    # is never a network input (h = 0 cells are accepted before the network)


def test_mlp_decide_reports_its_branches(tree):
    """Per-pair decisions: every branch the rule names occurs on a Plummer
    sphere, the band and fallback branches agree with the plain tests, and the
    network decides by its prediction. Inside the band l/d lies in
    [theta_lo, theta_hi), so an upper limit of 0.8 on input 3 (l/d) sends part
    of the band to the fallback; point cells reach the band only when
    theta_lo = 0 (otherwise the theta_lo test accepts them first)."""
    T = tree
    seen = set()
    f32 = np.float32
    for lo, fmax3 in ((0.45, 0.8), (0.0, np.inf)):
        net = _open_net()
        net["fmax"][3] = fmax3
        hi, fb, tau = 1.2, 0.7, 0.0
        for g in W.sample_indices(T.n_groups, 6, seed=9):
            gc = int(T.groups[g])
            for c in range(1, T.n_cells):
                op, br, y = T.mlp_decide(int(g), c, net, tau, lo, hi, fb)
                seen.add(br)
                args = (T.bmin[gc].astype(f32), T.bmax[gc].astype(f32), T.cube[c, :3].astype(f32),
                        f32(T.cube[c, 3]))
                if br == 0:
                    assert op and O.open_f32(*args, hi)
                elif br == 1:
                    assert not op and not O.open_f32(*args, lo)
                elif br == 2:
                    assert not op and T.cube[c, 3] == 0 and lo == 0.0
                elif br == 3:
                    assert op == O.open_f32(*args, fb) and T.mlp_features(int(g), c)[3] > fmax3
                else:
                    assert op == (not y < tau) and y != 0.0
    assert seen == {0, 1, 2, 3, 4}
    with pytest.raises(ValueError):
        T.mlp_decide(0, T.n_cells, net, tau, 0.45, 1.2, 0.7)


def test_mlp_decide_many_equals_single_decisions(tree):
    """The batched decision call gives each pair's single-call result, and the
    inputs it reports are the pair's features."""
    T = tree
    net = _open_net(6)
    net["fmax"][3] = 0.8
    rng = np.random.default_rng(1)
    g = rng.integers(0, T.n_groups, 400)
    c = rng.integers(1, T.n_cells, 400)
    op, br, y, f = T.mlp_decide_many(g, c, net, 0.0, 0.45, 1.2, 0.7, features=True)
    for k in range(400):
        assert (op[k], br[k], y[k]) == T.mlp_decide(int(g[k]), int(c[k]), net, 0.0, 0.45, 1.2, 0.7)
        if br[k] >= 3:
            np.testing.assert_array_equal(f[k], T.mlp_features(int(g[k]), int(c[k])))
    assert set(br.tolist()) >= {0, 1, 3, 4}
