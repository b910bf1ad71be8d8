"""GPU parity: the sm_103a walk + evaluation kernel against the FP64 CPU oracle.

Interaction lists must equal the oracle's bit for bit as multisets of cell
keys; accelerations must agree within 1e-5 relative RMS (FP32 evaluation vs
FP64 oracle on the same lists). Every call goes through the C ABI.
"""
import numpy as np
import pytest

import oracle as O
from paper_1005_5384_gb300 import octgrav as G
from paper_1005_5384_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_RMS = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()
    return torch


def _list_parity(pos, m, n_leaf, n_group, theta, ppl=2):
    T = G.Tree.build(pos, m, n_leaf, n_group)
    T.set_launch(ppl)
    R = O.Tree(pos, m, n_leaf, n_group)
    gl = T.debug_lists(theta, cap=max(4096, R.n_cells))
    info = T.item_info()
    okey = {int(R.key[c]): g for g, c in enumerate(R.groups)}
    checked = 0
    for k, (ck, lk) in enumerate(gl):
        g = okey[int(info["group_key"][k])]
        rc, rl = R.list_keys(g, theta)
        assert np.array_equal(ck, rc), (k, len(ck), len(rc))
        assert np.array_equal(lk, rl), (k, len(lk), len(rl))
        checked += 1
    assert checked == T.stats["n_items"]
    return T, R


@pytest.mark.parametrize("theta", [0.0, 0.5, 0.75, 1.2])
@pytest.mark.parametrize("n_group", [16, 64])
def test_lists_bit_exact_plummer(theta, n_group):
    pos, m = W.plummer(16384, seed=1)
    _list_parity(pos, m, 16, n_group, theta)


@pytest.mark.parametrize("ppl", [1, 2])
def test_lists_bit_exact_clustered(ppl):
    pos, m = W.clustered(20000, 8, seed=3)
    _list_parity(pos, m, 16, 48, 0.5, ppl)


def _force_parity(pos, m, n_leaf, n_group, eps, theta, ppl=2, G_=1.0):
    T = G.Tree.build(pos, m, n_leaf, n_group)
    T.set_launch(ppl)
    acc, pot = T.forces(eps, theta, G=G_)
    R = O.Tree(pos, m, n_leaf, n_group)
    ra, rp, _, _, _ = R.forces(eps, theta, G=G_)
    err = O.rel_rms(acc, ra)
    perr = float(np.linalg.norm(pot - rp) / np.linalg.norm(rp))
    assert err <= TOL_RMS, err
    assert perr <= TOL_RMS, perr
    return T, acc, pot


def test_forces_plummer_16k_matches_oracle_and_direct():
    pos, m = W.plummer(16384, seed=1)
    T, acc, pot = _force_parity(pos, m, 16, 16, 0.01, 0.5)
    ad, pd = O.direct(pos, m, 0.01)
    e = O.rel_err(acc, ad)
    assert np.median(e) < 1e-3
    c = T.interaction_counts()
    R = O.Tree(pos, m, 16, 16)
    _, _, npp, npc, _ = R.forces(0.01, 0.5)
    assert c["n_pp"] == int(npp.sum()) and c["n_pc"] == int(npc.sum())


@pytest.mark.parametrize("ppl,n_group", [(1, 16), (1, 32), (2, 64), (2, 48)])
def test_forces_lane_mappings(ppl, n_group):
    pos, m = W.plummer(12000, seed=7)
    _force_parity(pos, m, 16, n_group, 0.01, 0.6, ppl=ppl)


def test_forces_clustered_fp32_hard_case():
    """64 tight clusters, eps = 1e-3: separations ~1e-4 at |x| ~ 1."""
    pos, m = W.clustered(65536, 64, seed=3)
    _force_parity(pos, m, 16, 64, 0.001, 0.5)


def test_theta_zero_equals_direct_sum():
    pos, m = W.plummer(4096, seed=13)
    T = G.Tree.build(pos, m, 16, 16)
    acc, pot = T.forces(0.01, 0.0)
    ad, pd = O.direct(pos, m, 0.01)
    assert O.rel_rms(acc, ad) <= TOL_RMS
    assert float(np.linalg.norm(pot - pd) / np.linalg.norm(pd)) <= TOL_RMS


@pytest.mark.parametrize("n", [1, 2, 3, 17, 65, 129, 1000])
def test_ragged_and_tiny_inputs(n):
    pos, m = W.uniform_cube(n, seed=n)
    eps = 0.05
    acc, pot = G.forces(pos, m, eps, 0.7, n_leaf=1 if n < 20 else 4, n_group=4 if n < 20 else 8)
    if n == 1:
        assert np.all(acc == 0) and np.all(pot == 0)
        return
    ad, pd = O.direct(pos, m, eps)
    R = O.Tree(pos, m, 1 if n < 20 else 4, 4 if n < 20 else 8)
    ra, rp, _, _, _ = R.forces(eps, 0.7)
    assert O.rel_rms(acc, ra) <= TOL_RMS
    assert float(np.linalg.norm(pot - rp) / np.linalg.norm(rp)) <= TOL_RMS


def test_coincident_particles_and_split_items():
    """A max-depth leaf with 140 coincident particles is split over 3 warps."""
    rng = np.random.default_rng(5)
    pos = np.zeros((300, 3))
    pos[:140] = [0.3, 0.3, 0.3]
    pos[140:] = rng.random((160, 3))
    m = np.full(300, 1 / 300)
    T = G.Tree.build(pos, m, 4, 8)
    assert T.stats["max_group"] == 140
    acc, pot = T.forces(0.02, 0.5)
    R = O.Tree(pos, m, 4, 8)
    ra, rp, _, _, _ = R.forces(0.02, 0.5)
    assert O.rel_rms(acc, ra) <= TOL_RMS
    assert float(np.linalg.norm(pot - rp) / np.linalg.norm(rp)) <= TOL_RMS


def test_device_output_order_and_determinism(_cuda):
    torch = _cuda
    pos, m = W.plummer(30000, seed=2)
    T = G.Tree.build(pos, m, 16, 64)
    out = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    T.forces_device(0.01, 0.5, out)
    torch.cuda.synchronize()
    assert T.status() == G.OK
    a1 = out.cpu().numpy().copy()
    T.forces_device(0.01, 0.5, out)
    a2 = out.cpu().numpy()
    assert np.array_equal(a1, a2)                     # bitwise reproducible
    acc, pot = T.forces(0.01, 0.5)
    perm = T.perm()
    np.testing.assert_array_equal(acc[perm], a1[:, :3].astype(np.float64))
    np.testing.assert_array_equal(pot[perm], a1[:, 3].astype(np.float64))


def test_full_size_plummer_sampled_groups():
    """1,048,576-particle Plummer sphere at theta = 0.5 with N_group 64 (the
    benchmark's own configuration is in test_gpu_fullsize.py); the oracle
    evaluates a seeded sample of 400 groups."""
    pos, m = W.plummer(1 << 20, seed=1)
    T = G.Tree.build(pos, m, 16, 64)
    acc, pot = T.forces(0.01, 0.5)
    R = O.Tree(pos, m, 16, 64)
    gsel = np.unique(W.sample_indices(R.n_groups, 400, seed=9))
    ra, rp, _, _, _ = R.forces(0.01, 0.5, groups=gsel, counts=False)
    idx = np.concatenate([R.cell_members(int(R.groups[g])) for g in gsel])
    assert O.rel_rms(acc[idx], ra[idx]) <= TOL_RMS
    assert float(np.linalg.norm(pot[idx] - rp[idx]) / np.linalg.norm(rp[idx])) <= TOL_RMS
    samp = idx[:: max(1, len(idx) // 512)]
    ad, _ = O.direct(pos, m, 0.01, targets=samp)
    assert np.median(O.rel_err(acc[samp], ad)) < 1e-3


@pytest.mark.parametrize("stage", [0, 1, 2])
def test_staging_modes_agree_bitwise(_cuda, stage):
    """The three ways of staging cell records (per-record bulk copy, per-lane
    16-byte cp.async, TMA gather4) feed the same slots in the same order."""
    torch = _cuda
    pos, m = W.clustered(30000, 16, seed=8)
    T = G.Tree.build(pos, m, 16, 64)
    T.set_staging(stage)
    acc, pot = T.forces(0.005, 0.6)
    R = O.Tree(pos, m, 16, 64)
    ra, rp, _, _, _ = R.forces(0.005, 0.6)
    assert O.rel_rms(acc, ra) <= TOL_RMS
    T.set_staging(2)
    acc2, pot2 = T.forces(0.005, 0.6)
    assert np.array_equal(acc, acc2) and np.array_equal(pot, pot2)
    T.set_staging(stage)
    gl = T.debug_lists(0.6, cap=R.n_cells)
    info = T.item_info()
    okey = {int(R.key[c]): g for g, c in enumerate(R.groups)}
    for k in range(0, len(gl), 5):
        rc, rl = R.list_keys(okey[int(info["group_key"][k])], 0.6)
        assert np.array_equal(gl[k][0], rc) and np.array_equal(gl[k][1], rl)


def test_longest_first_order_changes_nothing_but_the_order(_cuda):
    torch = _cuda
    pos, m = W.plummer(60000, seed=12)
    T = G.Tree.build(pos, m, 16, 128)
    out = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(G.OctgravError) as e:
        T.balance()
    assert e.value.code == G.ERR_STATE
    T.forces_device(0.01, 0.5, out)
    torch.cuda.synchronize()
    ref = out.cpu().numpy().copy()
    c0 = T.interaction_counts()
    T.balance()
    out.zero_()
    T.forces_device(0.01, 0.5, out)
    torch.cuda.synchronize()
    assert T.status() == G.OK
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    assert T.interaction_counts() == c0
    for mode in (0, 2):  # tree order and most-particles-first: the same bits
        T.balance(mode)
        out.zero_()
        T.forces_device(0.01, 0.5, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    T.set_launch(1)  # new work items with their default order, results still right
    T.forces_device(0.01, 0.5, out)
    torch.cuda.synchronize()
    assert T.status() == G.OK
    T.balance(0)


def test_forced_stack_overflow_reports_err_stack(_cuda):
    """Failure injection without a fault: walks given 8 node-stack entries
    overflow, the launch reports ERR_STACK through the device status word, and
    the next launch on the same context is exact again."""
    pos, m = W.plummer(30000, seed=51)
    T = G.Tree.build(pos, m, 16, 64)
    ra, rp = T.forces(0.01, 0.5)
    T.set_fault(stack_cap=8)
    with pytest.raises(G.OctgravError) as e:
        T.forces(0.01, 0.5)
    assert e.value.code == G.ERR_STACK
    T.set_fault()
    a, p = T.forces(0.01, 0.5)
    assert np.array_equal(a, ra) and np.array_equal(p, rp)


def test_forced_wait_timeout_reports_err_timeout(_cuda):
    """Failure injection without a fault or a hang: in gather4 staging the first
    tile of one work item is never requested, so its bounded mbarrier wait
    (~1 s) runs out; the warp waits for its other copies and stops, the launch
    reports ERR_TIMEOUT, and the context stays usable."""
    import time

    pos, m = W.plummer(30000, seed=52)
    T = G.Tree.build(pos, m, 16, 64)
    T.set_staging(2)
    ra, rp = T.forces(0.01, 0.5)
    T.set_fault(drop_item=0)
    t0 = time.perf_counter()
    with pytest.raises(G.OctgravError) as e:
        T.forces(0.01, 0.5)
    assert e.value.code == G.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60
    T.set_fault()
    a, p = T.forces(0.01, 0.5)
    assert np.array_equal(a, ra) and np.array_equal(p, rp)
    with pytest.raises(G.OctgravError) as e:
        T.set_fault(drop_item=T.stats["n_items"])
    assert e.value.code == G.ERR_ARG


def test_small_capture_buffer_reports_err_list(_cuda):
    """The list-capture buffer is bounded on the device: a capacity of 4 entries
    per work item is exceeded and reported as ERR_LIST (the kernel writes only
    within the buffer); a large enough buffer then captures normally."""
    pos, m = W.plummer(8192, seed=53)
    T = G.Tree.build(pos, m, 16, 64)
    with pytest.raises(G.OctgravError) as e:
        T.debug_lists(0.5, cap=4)
    assert e.value.code == G.ERR_LIST
    assert len(T.debug_lists(0.5, cap=8192)) == T.stats["n_items"]


@pytest.mark.parametrize("shape", ["plane", "line", "two_points_and_a_cloud", "zero_masses", "far_offset"])
def test_degenerate_geometries(_cuda, shape):
    """Flat and one-dimensional systems (zero extent on some axes: boxes and
    cubes of zero thickness, distances along a single axis), a cloud with two
    heavy coincident pairs, a third of the particles massless (cells of zero
    mass take the cube centre as centre of mass), and a cloud of unit size
    10^4 away from the origin (FP32 absolute coordinates would keep ~1e-3 of
    its structure; the group-relative hi/lo coordinates keep it all): lists
    bit-exact and forces within 1e-5 of the oracle, GPU build identical to the
    host build."""
    rng = np.random.default_rng(60)
    n = 40000
    pos = rng.standard_normal((n, 3))
    if shape == "plane":
        pos[:, 2] = 0.0
    elif shape == "line":
        pos[:, 1] = 0.0
        pos[:, 2] = 0.0
    elif shape == "two_points_and_a_cloud":
        pos[:2] = [0.3, 0.3, 0.3]
        pos[2:4] = [-1.0, 0.5, 2.0]
    elif shape == "far_offset":
        pos += np.array([1.0e4, -1.0e4, 3.0e3])
    m = np.full(n, 1.0 / n)
    if shape == "two_points_and_a_cloud":
        m[:4] = 0.05
    elif shape == "zero_masses":
        m[::3] = 0.0
    T, R = _list_parity(pos, m, 16, 64, 0.6)
    acc, pot = T.forces(0.01, 0.6)
    ra, rp, _, _, _ = R.forces(0.01, 0.6)
    assert O.rel_rms(acc, ra) <= TOL_RMS
    assert float(np.linalg.norm(pot - rp) / np.linalg.norm(rp)) <= TOL_RMS
    acc_g, _ = G.forces_gpu(pos, m, 0.01, 0.6, 16, 64)
    assert np.array_equal(acc_g, acc)


@pytest.mark.parametrize("nparts,n,n_group,ppl", [(2, 16384, 16, 2), (4, 16384, 16, 2), (4, 16384, 128, 1),
                                                  (8, 16384, 128, 1), (16, 16384, 64, 2), (4, 200, 16, 2)])
def test_list_split_matches_unsplit_and_oracle(_cuda, nparts, n, n_group, ppl):
    """List split (a small system's work items walked by several warps, each
    evaluating a share of the lists): the same interaction counts as the
    unsplit launch, forces within FP32 rounding of it and within 1e-5 of the
    oracle, bitwise reproducible, and the same through a captured graph; from
    2 to 16 parts, 1 or 2 particles per lane, and a tree of 200 particles."""
    torch = _cuda
    pos, m = W.plummer(n, seed=1)
    T = G.Tree.build(pos, m, 16, n_group)
    T.set_launch(ppl)
    a1, p1 = T.forces(0.01, 0.5)
    c1 = T.interaction_counts()
    T.set_split(nparts)
    a2, p2 = T.forces(0.01, 0.5)
    c2 = T.interaction_counts()
    assert c1["n_pc"] == c2["n_pc"] and c1["n_pp"] == c2["n_pp"]
    assert O.rel_rms(a2, a1) <= 1e-6
    R = O.Tree(pos, m, 16, n_group)
    ra, rp, _, _, _ = R.forces(0.01, 0.5)
    assert O.rel_rms(a2, ra) <= TOL_RMS
    assert float(np.linalg.norm(p2 - rp) / np.linalg.norm(rp)) <= TOL_RMS
    a3, _ = T.forces(0.01, 0.5)
    assert np.array_equal(a2, a3)
    out = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        T.forces_device(0.01, 0.5, out, stream=st)
        st.synchronize()
        ref = out.clone()
        T.capture_graph(0.01, 0.5, out, stream=st)
        out.zero_()
        T.launch_graph(stream=st)
        st.synchronize()
    assert torch.equal(out, ref)
    with pytest.raises(G.OctgravError):
        T.set_split(0)


def test_list_split_on_a_batch(_cuda):
    """A split launch over many systems in one tree: every system equals its
    unsplit result within FP32 rounding and the interaction counts agree."""
    systems = W.ensemble(12, seed=9, n_min=300, n_max=5000)
    T = G.Tree.build_batch(systems, 16, 64)
    a1, _ = T.forces(0.01, 0.6)
    c1 = T.interaction_counts()
    T.set_split(4)
    a2, _ = T.forces(0.01, 0.6)
    c2 = T.interaction_counts()
    assert c1 == c2
    assert O.rel_rms(a2, a1) <= 1e-6
