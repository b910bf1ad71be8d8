"""Pins of the CPU FP64 oracle against facts that do not come from the oracle.

Each test checks the oracle against mathematics or a hand-worked case:
closed forms, symmetry, conservation, analytic profiles, brute force on tiny
inputs, convergence rates and hand-derived interaction lists. A dropped term,
a wrong sign or index or a transposed operand anywhere in the oracle fails at
least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1005_5384_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- O1 direct sum

def test_direct_three_body_golden():
    """Hand-worked Newtonian values (eps = 0) from tests/golden/three_body_line.txt."""
    rows = np.loadtxt(os.path.join(GOLDEN, "three_body_line.txt"))
    pos, m = rows[:, :3].copy(), rows[:, 3].copy()
    acc, pot = O.direct(pos, m, eps=0.0, nthreads=1)
    np.testing.assert_allclose(acc[:, 0], rows[:, 4] / rows[:, 5], rtol=1e-15, atol=0)
    np.testing.assert_array_equal(acc[:, 1:], 0.0)
    np.testing.assert_allclose(pot, rows[:, 6] / rows[:, 7], rtol=1e-15, atol=0)


@pytest.mark.parametrize("eps", [0.0, 0.3])
def test_direct_two_body_closed_form(eps):
    """a = G m r / (r^2 + eps^2)^{3/2}, phi = -G m / (r^2 + eps^2)^{1/2}."""
    x1 = np.array([0.3, -1.2, 2.0])
    r = np.array([1.5, 0.25, -0.75])
    pos = np.stack([x1, x1 + r])
    m = np.array([2.0, 0.7])
    G = 1.7
    acc, pot = O.direct(pos, m, eps=eps, G=G, nthreads=1)
    s2 = r @ r + eps * eps
    np.testing.assert_allclose(acc[0], G * m[1] * r / s2 ** 1.5, rtol=1e-14)
    np.testing.assert_allclose(acc[1], -G * m[0] * r / s2 ** 1.5, rtol=1e-14)
    np.testing.assert_allclose(pot, [-G * m[1] / math.sqrt(s2), -G * m[0] / math.sqrt(s2)], rtol=1e-14)


def test_direct_octahedron_symmetry():
    """A particle at the centre of a regular octahedron of equal masses feels no force."""
    R, eps = 1.3, 0.05
    pts = [[0, 0, 0]] + [[s * R if k == a else 0 for k in range(3)] for a in range(3) for s in (1, -1)]
    pos = np.array(pts, dtype=float) + np.array([0.4, -0.2, 7.0])
    m = np.array([0.5] + [1.25] * 6)
    acc, pot = O.direct(pos, m, eps=eps, nthreads=1)
    assert np.abs(acc[0]).max() < 1e-14
    assert pot[0] == pytest.approx(-6 * 1.25 / math.sqrt(R * R + eps * eps), rel=1e-14)


def test_direct_momentum_conservation():
    """Pairwise antisymmetry: sum_i m_i a_i = 0 to rounding."""
    pos, m = W.uniform_cube(700, seed=3)
    acc, _ = O.direct(pos, m, eps=0.01, nthreads=2)
    tot = np.abs((m[:, None] * acc).sum(0)).max()
    scale = (m[:, None] * np.abs(acc)).sum()
    assert tot / scale < 1e-13


def test_direct_plummer_analytic_profile():
    """Shell-averaged radial acceleration and potential of a Plummer sphere.

    Analytic (M = a = G = 1): a_r(r) = -r / (r^2 + 1)^{3/2}, phi(r) = -1/sqrt(r^2 + 1).
    Tolerance: Poisson noise of the sampled mass plus the O(eps^2) softening bias."""
    n = 16384
    pos, m = W.plummer(n, seed=21)
    eps = 1e-3
    r = np.linalg.norm(pos, axis=1)
    edges = np.quantile(r, np.linspace(0.05, 0.95, 10))
    idx = np.nonzero((r > edges[0]) & (r < edges[-1]))[0][::4]
    acc, pot = O.direct(pos, m, eps=eps, targets=idx)
    ar = (acc * pos[idx]).sum(1) / r[idx]
    rr = r[idx]
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (rr >= lo) & (rr < hi)
        rm = rr[sel]
        ana_a = (-rm / (rm * rm + 1) ** 1.5).mean()
        ana_p = (-1 / np.sqrt(rm * rm + 1)).mean()
        inner = np.mean(r < lo)
        noise = 4.0 / math.sqrt(max(1.0, inner * n)) + 1e-3
        assert abs(ar[sel].mean() / ana_a - 1) < noise
        assert abs(pot[sel].mean() / ana_p - 1) < 4.0 / math.sqrt(n) + 1e-3


# ---------------------------------------------------------------- O2/O3 tree

@pytest.fixture(scope="module")
def small_tree():
    pos, m = W.plummer(3000, seed=5)
    return O.Tree(pos, m, n_leaf=8, n_group=24)


def test_tree_partition_and_counts(small_tree):
    T = small_tree
    leaves = np.nonzero(T.leaf)[0]
    assert T.count[leaves].sum() == T.n
    members = np.concatenate([T.cell_members(c) for c in leaves])
    assert np.array_equal(np.sort(members), np.arange(T.n))
    for c in range(T.n_cells):
        kids = T.child[c][T.child[c] >= 0]
        if T.leaf[c]:
            assert len(kids) == 0
            assert T.count[c] <= T.n_leaf or T.depth[c] == T.max_depth
        else:
            assert T.count[c] > T.n_leaf
            assert T.count[kids].sum() == T.count[c]
            for k in kids:
                assert T.key[k] >> np.uint64(3) == T.key[c]
                assert T.depth[k] == T.depth[c] + 1


def test_tree_octant_geometry(small_tree):
    """Every member of a cell lies inside the cell's octree cube of side side/2^depth."""
    T = small_tree
    for c in range(0, T.n_cells, 7):
        L = int(T.depth[c])
        key = int(T.key[c])
        path = key ^ (1 << (3 * L))
        ijk = np.zeros(3)
        for lev in range(L):
            o = (path >> (3 * (L - 1 - lev))) & 7
            ijk = ijk * 2 + np.array([o & 1, (o >> 1) & 1, (o >> 2) & 1])
        s = T.side / 2 ** L
        lo = T.lo + ijk * s
        x = T.pos[T.cell_members(c)]
        assert np.all(x >= lo - 1e-12 * T.side) and np.all(x <= lo + s + 1e-12 * T.side)


def test_tree_moments(small_tree):
    """Mass, centre of mass, tight box, boundary cube and the parallel-axis theorem."""
    T = small_tree
    assert T.M[0] == pytest.approx(T.mass.sum(), rel=1e-14)
    np.testing.assert_allclose(T.com[0], (T.mass[:, None] * T.pos).sum(0) / T.mass.sum(), rtol=1e-12, atol=1e-14)
    for c in range(0, T.n_cells, 5):
        x = T.pos[T.cell_members(c)]
        np.testing.assert_array_equal(T.bmin[c], x.min(0))
        np.testing.assert_array_equal(T.bmax[c], x.max(0))
        ext = (x.max(0) - x.min(0)).max()
        assert T.cube[c, 3] == 0.5 * ext                       # half of the longest side
        np.testing.assert_array_equal(T.cube[c, :3], (x.min(0) + x.max(0)) * 0.5)
        kids = T.child[c][T.child[c] >= 0]
        if len(kids):
            Sp = np.zeros(6)
            for k in kids:
                d = T.com[k] - T.com[c]
                outer = np.array([d[0] * d[0], d[1] * d[1], d[2] * d[2], d[0] * d[1], d[0] * d[2], d[1] * d[2]])
                Sp += T.S[k] + T.M[k] * outer
            np.testing.assert_allclose(T.S[c], Sp, rtol=1e-11, atol=1e-14 * abs(T.S[c]).max())


def test_groups_cover_and_maximality(small_tree):
    T = small_tree
    covered = np.concatenate([T.cell_members(int(c)) for c in T.groups])
    assert np.array_equal(np.sort(covered), np.arange(T.n))
    for c in T.groups:
        assert T.leaf[c] or T.count[c] <= T.n_group
        p = T.parent[c]
        assert p < 0 or (T.count[p] > T.n_group and not T.leaf[p])
    # depth-first (key-path) order: member ranges are consecutive
    firsts = T.first[T.groups]
    assert np.all(np.diff(firsts) > 0)


def test_coincident_particles_reach_max_depth():
    pos = np.zeros((40, 3))
    pos[:30] = [0.25, 0.5, 0.75]
    pos[30:] = np.random.default_rng(0).random((10, 3))
    m = np.full(40, 1 / 40)
    T = O.Tree(pos, m, n_leaf=4)
    deep = np.nonzero(T.leaf & (T.count > 4))[0]
    assert len(deep) == 1 and T.depth[deep[0]] == O.MAX_DEPTH and T.count[deep[0]] == 30


# ---------------------------------------------------------------- O4 opening test

def test_opening_test_exact_cases():
    """Distance between box and cube; open iff side >= theta * distance; ties open."""
    gmin, gmax = [0, 0, 0], [1, 1, 1]
    # cube [3,5] x [0,1] x [0,1] (centre 4, h 1): d = 2, side 2
    c = [4.0, 0.5, 0.5]
    assert O.open_f32(gmin, gmax, c, 1.0, 0.5)          # 2 >= 1
    assert O.open_f32(gmin, gmax, c, 1.0, 1.0)          # 2 >= 2 (tie opens)
    assert not O.open_f32(gmin, gmax, c, 1.0, 1.0 + 1e-6)
    assert not O.open_f32(gmin, gmax, c, 1.0, 1.5)      # 2 < 3
    # below on every axis: cube [-4,-2]^3 -> d = sqrt(12)
    c = [-3.0, -3.0, -3.0]
    assert not O.open_f32(gmin, gmax, c, 1.0, 0.6)      # 2 < 0.6 * 3.46
    assert O.open_f32(gmin, gmax, c, 1.0, 0.57)         # 2 >= 0.57 * 3.46
    # overlap -> d = 0 -> always open, even theta huge
    assert O.open_f32(gmin, gmax, [1.2, 0.5, 0.5], 0.5, 100.0)
    # a point cell (h = 0) away from the box is always accepted
    assert not O.open_f32(gmin, gmax, [1.001, 0.5, 0.5], 0.0, 1e-3)
    # theta = 0 opens everything
    assert O.open_f32(gmin, gmax, [1e6, 1e6, 1e6], 1e-9, 0.0)


# ---------------------------------------------------------------- O5 walk

def _brute_lists(T, g, theta):
    """Independent characterisation: a cell joins a list iff every strict
    ancestor is opened; accepted -> cell list, opened leaf -> leaf list."""
    gc = T.groups[g]
    opened = np.zeros(T.n_cells, bool)
    for c in range(T.n_cells):
        opened[c] = O.open_f32(T.bmin[gc].astype(np.float32), T.bmax[gc].astype(np.float32),
                               T.cube[c, :3].astype(np.float32), np.float32(T.cube[c, 3]), theta)
    if T.leaf[0]:
        return np.array([], np.uint64), np.array([T.key[0]])
    cells, leaves = [], []
    for c in range(1, T.n_cells):
        a, ok = T.parent[c], True
        while a > 0:
            ok &= bool(opened[a])
            a = T.parent[a]
        if not ok:
            continue
        if not opened[c]:
            cells.append(T.key[c])
        elif T.leaf[c]:
            leaves.append(T.key[c])
    return np.sort(np.array(cells, np.uint64)), np.sort(np.array(leaves, np.uint64))


@pytest.mark.parametrize("theta", [0.0, 0.4, 0.9])
def test_walk_matches_brute_force(theta):
    pos, m = W.plummer(300, seed=9)
    T = O.Tree(pos, m, n_leaf=4, n_group=8)
    for g in range(0, T.n_groups, max(1, T.n_groups // 15)):
        ck, lk = T.list_keys(g, theta)
        bc, bl = _brute_lists(T, g, theta)
        assert np.array_equal(ck, bc) and np.array_equal(lk, bl)


def test_walk_lists_cover_every_particle_once():
    pos, m = W.clustered(4000, 8, seed=2)
    T = O.Tree(pos, m, n_leaf=8, n_group=16)
    for g in range(0, T.n_groups, 37):
        cells, leaves = T.lists(g, 0.6)
        mem = np.concatenate([T.cell_members(int(c)) for c in np.concatenate([cells, leaves])])
        assert np.array_equal(np.sort(mem), np.arange(T.n))
        # the group's own particles are always among the leaf-list members
        own = T.cell_members(int(T.groups[g]))
        assert np.isin(own, np.concatenate([T.cell_members(int(c)) for c in leaves])).all()


def test_walk_golden_two_clusters():
    path = os.path.join(GOLDEN, "two_clusters_lists.txt")
    pts, cases = [], []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("@"):
            head, cells, leaves = line[1:].split("|")
            gk, th = head.split()
            cases.append((int(gk), float(th), sorted(int(v) for v in cells.split()),
                          sorted(int(v) for v in leaves.split())))
        else:
            pts.append([float(v) for v in line.split()])
    pts = np.array(pts)
    T = O.Tree(pts[:, :3].copy(), pts[:, 3].copy(), n_leaf=1, n_group=1)
    gkeys = [int(k) for k in T.key[T.groups]]
    for gk, th, cells, leaves in cases:
        ck, lk = T.list_keys(gkeys.index(gk), th)
        assert [int(v) for v in ck] == cells and [int(v) for v in lk] == leaves


# ---------------------------------------------------------------- O6 evaluation

def _cell_of(pts, ms):
    M = ms.sum()
    com = (ms[:, None] * pts).sum(0) / M
    y = pts - com
    S = np.array([(ms * y[:, 0] * y[:, 0]).sum(), (ms * y[:, 1] * y[:, 1]).sum(), (ms * y[:, 2] * y[:, 2]).sum(),
                  (ms * y[:, 0] * y[:, 1]).sum(), (ms * y[:, 0] * y[:, 2]).sum(), (ms * y[:, 1] * y[:, 2]).sum()])
    return com, M, S


def test_cell_field_convergence_orders():
    """Relative error of the expansion vs the exact member sum falls as (l/d)^3;
    without the second moments (monopole only) it falls as (l/d)^2."""
    rng = np.random.default_rng(4)
    pts = rng.random((40, 3)) - 0.5
    ms = 0.5 + rng.random(40)
    com, M, S = _cell_of(pts, ms)
    direction = np.array([0.48, 0.6, 0.64])
    ds = np.array([8.0, 16.0, 32.0, 64.0])
    e_q, e_m = [], []
    for d in ds:
        x = com + d * direction
        a_ex, _ = O.direct(np.vstack([pts, x]), np.append(ms, 0.0), eps=0.0, targets=[40])
        a_q, _ = O.cell_field(com, M, S, x, 0.0)
        a_m, _ = O.cell_field(com, M, np.zeros(6), x, 0.0)
        e_q.append(np.linalg.norm(a_q - a_ex[0]) / np.linalg.norm(a_ex[0]))
        e_m.append(np.linalg.norm(a_m - a_ex[0]) / np.linalg.norm(a_ex[0]))
    slope_q = np.polyfit(np.log(ds), np.log(e_q), 1)[0]
    slope_m = np.polyfit(np.log(ds), np.log(e_m), 1)[0]
    assert -3.3 < slope_q < -2.7
    assert -2.3 < slope_m < -1.7


def test_cell_field_is_minus_gradient_of_potential():
    rng = np.random.default_rng(8)
    pts = rng.random((12, 3))
    ms = rng.random(12) + 0.1
    com, M, S = _cell_of(pts, ms)
    x = com + np.array([2.5, -1.0, 1.7])
    eps, h = 0.3, 1e-5
    a, _ = O.cell_field(com, M, S, x, eps, G=2.0)
    grad = np.zeros(3)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        grad[k] = (O.cell_field(com, M, S, x + e, eps, 2.0)[1] - O.cell_field(com, M, S, x - e, eps, 2.0)[1]) / (2 * h)
    np.testing.assert_allclose(a, -grad, rtol=1e-8)


def test_cell_field_eps0_matches_traceless_quadrupole():
    """With eps = 0: a = -M y/r^3 + Q y/r^5 - (5/2)(y.Q.y) y/r^7, Q = 3S - tr(S) I;
    phi = -M/r - (1/2) y.Q.y / r^5."""
    rng = np.random.default_rng(1)
    pts = rng.random((9, 3))
    ms = rng.random(9) + 0.2
    com, M, S6 = _cell_of(pts, ms)
    S = np.array([[S6[0], S6[3], S6[4]], [S6[3], S6[1], S6[5]], [S6[4], S6[5], S6[2]]])
    Q = 3 * S - np.trace(S) * np.eye(3)
    x = com + np.array([-3.0, 2.0, 4.0])
    y = x - com
    r = np.linalg.norm(y)
    a_ref = -M * y / r**3 + Q @ y / r**5 - 2.5 * (y @ Q @ y) * y / r**7
    p_ref = -M / r - 0.5 * (y @ Q @ y) / r**5
    a, p = O.cell_field(com, M, S6, x, 0.0)
    np.testing.assert_allclose(a, a_ref, rtol=1e-13)
    assert p == pytest.approx(p_ref, rel=1e-13)


# ---------------------------------------------------------------- whole tree

def test_theta_zero_tree_equals_direct_sum():
    """theta = 0 opens every cell, so the tree reduces to the direct sum."""
    pos, m = W.plummer(2000, seed=13)
    T = O.Tree(pos, m, n_leaf=16)
    acc, pot, npp, npc, _ = T.forces(0.01, 0.0)
    ad, pd = O.direct(pos, m, 0.01)
    assert O.rel_rms(acc, ad) < 1e-13
    np.testing.assert_allclose(pot, pd, rtol=1e-13)
    assert np.all(npc == 0) and np.all(npp == T.n - 1)


def test_error_scales_as_theta_to_the_fourth():
    """Sec. 3.1 fits the median relative error as ~theta^4 on its galaxy model.

    The expansion stops after the quadrupole, so each accepted cell leaves a
    relative error of order (l/r)^3 <= theta^3 (r >= d). The fitted log-log
    slope must therefore be steep (between 2.5 and 4.5): a monopole-only
    evaluation would give ~2, a broken opening test a flat curve."""
    pos, m = W.plummer(16384, seed=1)
    T = O.Tree(pos, m, n_leaf=16)
    samp = W.sample_indices(T.n, 1500, seed=2)
    ad, _ = O.direct(pos, m, 0.01, targets=samp)
    thetas = np.array([0.3, 0.4, 0.5, 0.6, 0.7])
    med = []
    for th in thetas:
        acc, _, _, _, _ = T.forces(0.01, th, counts=False)
        med.append(np.median(O.rel_err(acc[samp], ad)))
    slope = np.polyfit(np.log(thetas), np.log(med), 1)[0]
    assert 2.5 < slope < 4.5, (slope, med)
    assert med[2] < 1e-3


def test_tree_momentum_is_small():
    pos, m = W.plummer(8192, seed=4)
    T = O.Tree(pos, m, n_leaf=16)
    acc, _, _, _, _ = T.forces(0.01, 0.5)
    assert np.abs((m[:, None] * acc).sum(0)).max() / (m[:, None] * np.abs(acc)).sum() < 1e-3


def test_group_subset_matches_full_run():
    pos, m = W.plummer(5000, seed=6)
    T = O.Tree(pos, m, n_leaf=16, n_group=32)
    acc, pot, _, _, _ = T.forces(0.01, 0.5)
    gsel = np.arange(3, T.n_groups, 11)
    acc2, pot2, _, _, _ = T.forces(0.01, 0.5, groups=gsel)
    idx = np.concatenate([T.cell_members(int(T.groups[g])) for g in gsel])
    np.testing.assert_array_equal(acc2[idx], acc[idx])
    np.testing.assert_array_equal(pot2[idx], pot[idx])
