"""The octree built on the GPU against the host FP64 build and the oracle.

The GPU build runs the same steps as the host build (Sec. 2.1: root cube,
Morton keys, stable sort, level-by-level split, bottom-up moments, groups,
work items) with the same FP64 operations in the same order, so every array
must come out identical bit for bit; the forces of the two trees must then be
identical too (the walk kernel is deterministic per particle). The GPU-built
tree is also checked against the oracle directly, and on the edge cases of the
build: one particle, coincident particles (depth limit), tiny and multi-chunk
systems in a batch, a cell capacity that has to grow, invalid inputs.
"""
import numpy as np
import pytest

import oracle as O
from paper_1005_5384_gb300 import octgrav as G
from paper_1005_5384_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()
    return t


def _bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint8)


def _assert_same_tree(A, B):
    assert A.stats == B.stats
    assert np.array_equal(A.perm(), B.perm())
    assert np.array_equal(A.cell_keys(), B.cell_keys())
    pa, pb = A.cell_props(), B.cell_props()
    for k in pa:
        assert np.array_equal(_bits(pa[k]), _bits(pb[k])), k
    ia, ib = A.item_info(), B.item_info()
    for k in ia:
        assert np.array_equal(ia[k], ib[k]), k


def _device_forces(torch, T, eps, theta):
    out = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    T.forces_device(eps, theta, out)
    torch.cuda.synchronize()
    assert T.status() == G.OK
    return out.cpu().numpy()


def _coincident(n):
    return np.tile([[0.25, -0.5, 0.125]], (n, 1)), np.full(n, 1.0 / n)


def _clumps():
    """Clumps of coincident particles whose sizes sit on the work-item cut's bounds."""
    counts = [32, 33, 48, 49, 56, 64, 65, 80, 81]
    centres = np.random.default_rng(8).random((len(counts), 3))
    pos = np.concatenate([np.tile(c, (k, 1)) for c, k in zip(centres, counts)])
    return pos, np.full(len(pos), 1.0 / len(pos))


CASES = {
    "plummer_16k": (lambda: W.plummer(16384, seed=1), 16, 16, 0.01),
    "plummer_100k_ng64": (lambda: W.plummer(100000, seed=2), 16, 64, 0.01),
    "plummer_262k_ng256": (lambda: W.plummer(262144, seed=3), 16, 256, 0.01),
    "clustered_200k": (lambda: W.clustered(200000, 16, seed=4), 16, 64, 0.001),
    "sphere_disc_131k": (lambda: W.sphere_disc(131072, seed=5), 16, 64, 0.01),
    "uniform_nleaf1": (lambda: W.uniform_cube(50000, seed=6), 1, 8, 0.01),
    "one_particle": (lambda: (np.array([[0.3, 0.2, 0.1]]), np.array([1.0])), 1, 1, 0.01),
    "two_coincident": (lambda: _coincident(2), 1, 1, 0.01),
    "coincident_100": (lambda: _coincident(100), 4, 8, 0.01),
    "clumps_at_item_bounds": (_clumps, 4, 4, 0.01),
    "ragged_37": (lambda: W.plummer(37, seed=7), 4, 8, 0.01),
    "chunk_edges_8193": (lambda: W.plummer(8193, seed=8), 16, 32, 0.01),
    "galaxy_60k": (lambda: W.galaxy(60000, seed=9), 16, 64, 0.01),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_gpu_build_equals_host_build(torch, name):
    make, n_leaf, n_group, eps = CASES[name]
    pos, m = make()
    A = G.Tree.build(pos, m, n_leaf, n_group)
    B = G.Tree.build_gpu(pos, m, n_leaf, n_group)
    _assert_same_tree(A, B)
    fa = _device_forces(torch, A, eps, 0.6)
    fb = _device_forces(torch, B, eps, 0.6)
    assert np.array_equal(_bits(fa), _bits(fb))


def test_gpu_built_tree_matches_oracle(torch):
    pos, m = W.plummer(16384, seed=11)
    T = G.Tree.build_gpu(pos, m, 16, 32)
    R = O.Tree(pos, m, 16, 32)
    assert T.stats["n_cells"] == R.n_cells and T.stats["n_groups"] == R.n_groups
    k = T.cell_keys()
    assert np.array_equal(np.sort(k), np.sort(R.key))
    acc, pot = T.forces(0.01, 0.5)
    ra, rp, _, _, _ = R.forces(0.01, 0.5)
    assert O.rel_rms(acc, ra) <= 1e-5
    assert np.linalg.norm(pot - rp) / np.linalg.norm(rp) <= 1e-5


def test_galaxy_forces_match_oracle(torch):
    pos, m = W.galaxy(30000, seed=10)
    T = G.Tree.build_gpu(pos, m, 16, 64)
    acc, pot = T.forces(0.01, 0.5)
    R = O.Tree(pos, m, 16, 64)
    ra, rp, _, _, _ = R.forces(0.01, 0.5)
    assert O.rel_rms(acc, ra) <= 1e-5
    assert np.linalg.norm(pot - rp) / np.linalg.norm(rp) <= 1e-5


def test_batch_gpu_build_equals_host_batch(torch):
    sizes = (300, 1000, 17, 1, 2 * 4096 + 5, 4096, 2, 65)
    systems = [W.plummer(n, seed=20 + s) for s, n in enumerate(sizes)]
    A = G.Tree.build_batch(systems, 8, 32)
    pos = np.concatenate([p for p, _ in systems])
    m = np.concatenate([q for _, q in systems])
    off = np.concatenate([[0], np.cumsum(sizes)])
    B = G.Tree.build_gpu(pos, m, 8, 32, offsets=off)
    _assert_same_tree(A, B)
    fa = _device_forces(torch, A, 0.01, 0.7)
    fb = _device_forces(torch, B, 0.01, 0.7)
    assert np.array_equal(_bits(fa), _bits(fb))


def test_ensemble_gpu_build_equals_host_batch(torch):
    systems = W.ensemble(256, seed=4)
    A = G.Tree.build_batch(systems, 16, 64)
    pos = np.concatenate([p for p, _ in systems])
    m = np.concatenate([q for _, q in systems])
    off = np.concatenate([[0], np.cumsum([len(q) for _, q in systems])])
    B = G.Tree.build_gpu(pos, m, 16, 64, offsets=off)
    _assert_same_tree(A, B)
    assert np.array_equal(_bits(_device_forces(torch, A, 0.01, 0.6)), _bits(_device_forces(torch, B, 0.01, 0.6)))


def test_cell_capacity_grows(torch, monkeypatch):
    pos, m = W.plummer(60000, seed=12)
    monkeypatch.setenv("OCTGRAV_GPU_CELL_CAP", "64")
    B = G.Tree.build_gpu(pos, m, 16, 64)
    monkeypatch.delenv("OCTGRAV_GPU_CELL_CAP")
    A = G.Tree.build(pos, m, 16, 64)
    _assert_same_tree(A, B)


@pytest.mark.parametrize("ppl", [1, 2])
def test_work_items_rebuilt_on_the_device(torch, ppl):
    pos, m = W.plummer(50000, seed=13)
    A = G.Tree.build(pos, m, 16, 128)
    B = G.Tree.build_gpu(pos, m, 16, 128)
    B.item_info()  # host images made before the change must not go stale
    A.set_launch(ppl)
    B.set_launch(ppl)
    _assert_same_tree(A, B)
    assert np.array_equal(_bits(_device_forces(torch, A, 0.01, 0.5)), _bits(_device_forces(torch, B, 0.01, 0.5)))


def test_one_shot_gpu_call_equals_host_path(torch):
    pos, m = W.plummer(70000, seed=14)
    acc, pot = G.forces(pos, m, 0.01, 0.5, 16, 64)
    pin_x = torch.from_numpy(pos.copy()).pin_memory()
    pin_m = torch.from_numpy(m.copy()).pin_memory()
    out_a = torch.zeros((len(m), 3), dtype=torch.float64).pin_memory()
    out_p = torch.zeros(len(m), dtype=torch.float64).pin_memory()
    for _ in range(2):  # the second call reuses the cached device buffers
        a2, p2 = G.forces_gpu(pin_x.numpy(), pin_m.numpy(), 0.01, 0.5, 16, 64, out=(out_a.numpy(), out_p.numpy()))
        assert np.array_equal(_bits(acc), _bits(a2)) and np.array_equal(_bits(pot), _bits(p2))
    a3, p3 = G.forces_gpu(pos, m, 0.01, 0.5, 16, 64)  # pageable buffers
    assert np.array_equal(_bits(acc), _bits(a3)) and np.array_equal(_bits(pot), _bits(p3))


def test_one_shot_host_call_across_sizes(torch):
    """The host-build one-shot call keeps its host arrays between calls and
    starts the particle upload during the build: calls of growing and
    shrinking N (ragged, not multiples of 4) equal the tree path bit for bit."""
    for n, seed in ((50001, 31), (3, 32), (120003, 33), (20000, 34)):
        pos, m = W.plummer(n, seed=seed)
        T = G.Tree.build(pos, m, 16, 64)
        ra, rp = T.forces(0.01, 0.5)
        pin_x = torch.from_numpy(pos.copy()).pin_memory()
        pin_m = torch.from_numpy(m.copy()).pin_memory()
        out_a = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
        out_p = torch.zeros(n, dtype=torch.float64).pin_memory()
        a1, p1 = G.forces(pin_x.numpy(), pin_m.numpy(), 0.01, 0.5, 16, 64, out=(out_a.numpy(), out_p.numpy()))
        a2, p2 = G.forces(pos, m, 0.01, 0.5, 16, 64)  # pageable buffers
        for a, p in ((a1, p1), (a2, p2)):
            assert np.array_equal(_bits(a), _bits(ra)) and np.array_equal(_bits(p), _bits(rp))


def test_one_shot_calls_from_threads(torch):
    """Each calling thread has its own host arrays and device buffers: four
    threads calling both one-shot entry points at once get the single-thread
    results bit for bit, and their device buffers are released when they end."""
    import threading

    pos, m = W.plummer(40000, seed=41)
    ra, rp = G.forces(pos, m, 0.01, 0.5, 16, 64)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    results = [None] * 4
    errors = []

    def work(k):
        try:
            torch.cuda.set_device(0)
            out = []
            for _ in range(3):
                out += [G.forces(pos, m, 0.01, 0.5, 16, 64), G.forces_gpu(pos, m, 0.01, 0.5, 16, 64)]
            results[k] = out
        except Exception as e:  # reported below, on the main thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for out in results:
        for a, p in out:
            assert np.array_equal(_bits(a), _bits(ra)) and np.array_equal(_bits(p), _bits(rp))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)


def test_one_shot_copy_fallback_equals_pull(torch, monkeypatch):
    """With OCTGRAV_HOST_PULL=0 the one-shot call uploads with cudaMemcpyAsync
    instead of pulling pageable memory by kernel: the same results. (The
    setting is read when a thread's device buffers are first used, so the call
    runs on a new thread.)"""
    import threading

    pos, m = W.plummer(30001, seed=42)
    ra, rp = G.forces(pos, m, 0.01, 0.5, 16, 64)
    monkeypatch.setenv("OCTGRAV_HOST_PULL", "0")
    out = {}
    t = threading.Thread(target=lambda: out.update(r=G.forces(pos, m, 0.01, 0.5, 16, 64)))
    t.start()
    t.join()
    a, p = out["r"]
    assert np.array_equal(_bits(a), _bits(ra)) and np.array_equal(_bits(p), _bits(rp))


def test_oneshot_phases(torch):
    """The one-shot host-build call reports where its time went: every phase
    measured, the host phases adding up to the host build, the device phases
    and the build within the whole call."""
    pos, m = W.plummer(200000, seed=43)
    G.forces(pos, m, 0.01, 0.5, 16, 64)
    ph = G.oneshot_phases()
    assert list(ph) == list(G.ONESHOT_PHASES)
    assert all(v >= 0 for v in ph.values())
    host = sum(ph[k] for k in G.ONESHOT_PHASES[:8])
    assert host <= ph["host_build"] * 1.05 + 0.05
    assert ph["device_walk_eval"] > 0 and ph["host_build"] + ph["device_walk_eval"] <= ph["call"] * 1.05 + 0.05


def test_device64_outputs_in_input_order(torch):
    pos, m = W.plummer(30000, seed=15)
    for T in (G.Tree.build(pos, m, 16, 64), G.Tree.build_gpu(pos, m, 16, 64)):
        acc, pot = T.forces(0.01, 0.5)
        da = torch.empty((T.n, 3), dtype=torch.float64, device="cuda")
        dp = torch.empty(T.n, dtype=torch.float64, device="cuda")
        T.forces_device64(0.01, 0.5, da, dp)
        assert T.status() == G.OK
        assert np.array_equal(da.cpu().numpy(), acc) and np.array_equal(dp.cpu().numpy(), pot)


def test_invalid_inputs_are_reported(torch):
    pos, m = W.plummer(5000, seed=16)
    bad = pos.copy()
    bad[1234, 1] = np.nan
    with pytest.raises(G.OctgravError) as e:
        G.Tree.build_gpu(bad, m)
    assert e.value.code == G.ERR_NONFINITE
    neg = m.copy()
    neg[17] = -1.0
    with pytest.raises(G.OctgravError) as e:
        G.Tree.build_gpu(pos, neg)
    assert e.value.code == G.ERR_NONFINITE
    with pytest.raises(G.OctgravError) as e:
        G.Tree.build_gpu(pos, m, 16, 8)
    assert e.value.code == G.ERR_ARG
    with pytest.raises(G.OctgravError) as e:
        G.Tree.build_gpu(pos, m, 16, 16, offsets=[0, 3000, 3000, 5000])
    assert e.value.code == G.ERR_ARG
    # the library still works after the refusals
    T = G.Tree.build_gpu(pos, m, 16, 16)
    assert T.stats["n"] == 5000


def test_full_size_build_equals_host(torch):
    pos, m = W.plummer(1 << 20, seed=1)
    A = G.Tree.build(pos, m, 16, 512)
    B = G.Tree.build_gpu(pos, m, 16, 512)
    _assert_same_tree(A, B)


@pytest.mark.parametrize("case", ["clustered_8M_deep", "plummer_16M"])
def test_large_builds_equal_host(torch, case):
    if case == "clustered_8M_deep":
        pos, m = W.clustered(1 << 23, 256, seed=21, rs_min=1e-4, rs_max=1e-3)
    else:
        pos, m = W.plummer(1 << 24, seed=22)
    A = G.Tree.build(pos, m, 16, 256)
    B = G.Tree.build_gpu(pos, m, 16, 256)
    assert A.stats == B.stats
    assert np.array_equal(A.perm(), B.perm())
    assert np.array_equal(A.cell_keys(), B.cell_keys())
    pa, pb = A.cell_props(), B.cell_props()
    for k in ("M", "com", "S", "cube"):
        kk = {"M": "mass"}.get(k, k)
        assert np.array_equal(_bits(pa[kk]), _bits(pb[kk])), k


def test_level_cap_from_a_shallow_tree_is_lifted_for_a_deep_one(torch):
    # the one-shot call caches its buffers and caps the next level loop at the
    # previous depth + 2; a much deeper system of the same size must still come out right
    n = 50000
    shallow = W.uniform_cube(n, seed=31)
    deep = W.clustered(n, 8, seed=32, rs_min=1e-5, rs_max=1e-4)
    G.forces_gpu(*shallow, 0.01, 0.5, 16, 64)
    acc, pot = G.forces_gpu(*deep, 1e-6, 0.5, 16, 64)
    ra, rp = G.Tree.build(*deep, 16, 64).forces(1e-6, 0.5)
    assert np.array_equal(_bits(acc), _bits(ra)) and np.array_equal(_bits(pot), _bits(rp))
    assert G.Tree.build(*deep, 16, 64).stats["depth"] > G.Tree.build(*shallow, 16, 64).stats["depth"] + 2


def test_refit_at_the_same_positions_is_the_same_tree(torch):
    pos, m = W.plummer(40000, seed=41)
    B = G.Tree.build_gpu(pos, m, 16, 64)
    keys, props, info = B.cell_keys(), B.cell_props(), B.item_info()
    f0 = _device_forces(torch, B, 0.01, 0.5)
    B.refit(pos, m)
    assert np.array_equal(B.cell_keys(), keys)
    p1 = B.cell_props()
    for k in props:
        assert np.array_equal(_bits(p1[k]), _bits(props[k])), k
    for k in info:
        assert np.array_equal(B.item_info()[k], info[k]), k
    assert np.array_equal(_bits(_device_forces(torch, B, 0.01, 0.5)), _bits(f0))


def test_refit_recomputes_boxes_and_moments_from_the_new_positions(torch):
    pos, m = W.plummer(20000, seed=42)
    rng = np.random.default_rng(1)
    pos1 = pos + 0.01 * rng.standard_normal(pos.shape)
    m1 = m * (1.0 + 0.1 * rng.random(m.shape))
    B = G.Tree.build_gpu(pos, m, 16, 64)
    B.refit(pos1, m1)
    perm = B.perm()
    props = B.cell_props()
    x = pos1[perm]
    mm = m1[perm]
    keys = B.cell_keys()
    cnt = props["count"]
    # first particle (tree position) of each cell: a child starts where its parent
    # starts plus the counts of its earlier siblings (children ascend by octant)
    first = np.zeros(B.stats["n_cells"], np.int64)
    depth = np.floor(np.log2(keys.astype(np.float64)) / 3).astype(int)
    where = {int(k): c for c, k in enumerate(keys)}
    for L in range(1, depth.max() + 1):
        for c in np.nonzero(depth == L)[0]:
            parent = where[int(keys[c] >> np.uint64(3))]
            base = int(keys[parent]) << 3
            first[c] = first[parent] + sum(int(cnt[where[base | o]]) for o in range(int(keys[c]) & 7)
                                           if (base | o) in where)
    for c in rng.choice(B.stats["n_cells"], 300, replace=False):
        sl = slice(first[c], first[c] + cnt[c])
        xs, ms = x[sl], mm[sl]
        assert np.array_equal(props["bmin"][c], xs.min(0)) and np.array_equal(props["bmax"][c], xs.max(0))
        M = ms.sum()
        com = (ms[:, None] * xs).sum(0) / M
        y = xs - com
        S = np.einsum("i,ij,ik->jk", ms, y, y)
        assert abs(props["mass"][c] - M) <= 1e-13 * M
        assert np.allclose(props["com"][c], com, rtol=0, atol=1e-12 * (1 + np.abs(com).max()))
        s6 = np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]])
        assert np.allclose(props["S"][c], s6, rtol=1e-10, atol=1e-14 * max(1e-300, np.abs(s6).max()))
    # the refitted tree still gives accurate forces
    acc, _ = B.forces(0.01, 0.5)
    samp = W.sample_indices(len(m1), 400, seed=3)
    ad, _ = G.direct(pos1, m1, 0.01, targets=samp)
    assert np.median(G.rel_err(acc[samp], ad)) < 5e-4


def test_refit_refusals(torch):
    pos, m = W.plummer(5000, seed=43)
    with pytest.raises(G.OctgravError) as e:
        G.Tree.build(pos, m).refit(pos, m)
    assert e.value.code == G.ERR_STATE
    B = G.Tree.build_gpu(pos, m)
    bad = pos.copy()
    bad[7, 0] = np.inf
    with pytest.raises(G.OctgravError) as e:
        B.refit(bad, m)
    assert e.value.code == G.ERR_NONFINITE


def _runs(info):
    k = info["group_key"]
    starts = np.flatnonzero(np.r_[True, k[1:] != k[:-1]])
    return starts, np.r_[starts[1:], len(k)]


def test_learned_criterion_keeps_rests_whole(torch):
    """Setting a learned criterion cuts the items again without the 32 + rest
    split (one item per 33..48-particle rest), on the host-built and the
    GPU-built tree alike (the same items, byte for byte); a new record keeps
    them; clearing the criterion restores the split items; a graph captured
    before is dropped; the forces of the plain criterion are unchanged."""
    import oracle.mlp as M
    pos, m = W.plummer(30000, seed=12)
    A = G.Tree.build(pos, m, 16, 128)
    B = G.Tree.build_gpu(pos, m, 16, 128)
    plain = A.item_info()
    f0 = _device_forces(torch, B, 0.01, 0.6)
    s = torch.cuda.Stream()
    out = torch.empty((B.n, 4), dtype=torch.float32, device="cuda")
    B.capture_graph(0.01, 0.6, out, stream=s)
    rec = np.concatenate([np.zeros(12), np.ones(12), np.full(12, -1e3), np.full(12, 1e3), M.init(2)]).astype(np.float32)
    for T in (A, B):
        T.set_criterion(rec, tau=-3.0, theta_lo=0.5, theta_hi=1.0, theta_fb=0.7)
    ia, ib = A.item_info(), B.item_info()
    for k in ia:
        assert np.array_equal(ia[k], ib[k]), k
    assert A.stats == B.stats and A.stats["n_items"] < len(plain["count"])
    for a, b in zip(*_runs(ia)):
        c = int(ia["count"][a:b].sum())
        assert b - a == (c + 63) // 64 and ia["count"][a:b].max() <= 64
    with pytest.raises(G.OctgravError) as e:
        B.launch_graph(stream=s)
    assert e.value.code == G.ERR_STATE
    B.set_criterion(rec, tau=-2.0, theta_lo=0.5, theta_hi=1.0, theta_fb=0.7)
    assert np.array_equal(B.item_info()["count"], ib["count"])
    for T in (A, B):
        T.set_criterion(None)
        back = T.item_info()
        for k in plain:
            assert np.array_equal(back[k], plain[k]), k
    assert np.array_equal(_device_forces(torch, B, 0.01, 0.6), f0)

