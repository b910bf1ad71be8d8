"""CPU-only checks of the C-ABI library: it loads, exports every symbol the
header declares, validates its arguments without touching a GPU, and its host
FP64 octree equals the oracle's tree cell for cell."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1005_5384_gb300 import octgrav as G
from paper_1005_5384_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "octgrav.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(octgrav_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = G.load()
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(G.exported_symbols())
    assert G.version() >= 10000


@pytest.mark.parametrize("n,n_leaf,n_group", [(1, 1, 1), (2, 1, 1), (37, 4, 8), (3000, 8, 24), (20000, 16, 64)])
def test_host_tree_equals_oracle_tree(n, n_leaf, n_group):
    pos, m = W.plummer(n, seed=n + 3) if n > 2 else (np.array([[0.0, 0, 0], [1, 2, 3]])[:n], np.ones(n))
    T = G.Tree.build(pos, m, n_leaf, n_group)
    R = O.Tree(pos, m, n_leaf, n_group)
    k = T.cell_keys()
    assert T.stats["n_cells"] == R.n_cells and T.stats["n_leaves"] == R.n_leaves
    assert T.stats["n_groups"] == R.n_groups
    ol, oo = np.argsort(k), np.argsort(R.key)
    assert np.array_equal(k[ol], R.key[oo])
    p = T.cell_props()
    # boxes and cubes are exact min/max and x0.5 results: bit-identical
    assert np.array_equal(p["bmin"][ol], R.bmin[oo]) and np.array_equal(p["bmax"][ol], R.bmax[oo])
    assert np.array_equal(p["cube"][ol], R.cube[oo])
    assert np.array_equal(p["count"][ol], R.count[oo])
    # moments: parallel-axis combination vs direct sums, rounding only
    np.testing.assert_allclose(p["mass"][ol], R.M[oo], rtol=1e-11)
    np.testing.assert_allclose(p["com"][ol], R.com[oo], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(p["S"][ol], R.S[oo], rtol=1e-9, atol=1e-13 * max(1e-300, abs(R.S).max()))
    info = T.item_info()
    assert np.array_equal(np.unique(info["group_key"]), np.sort(R.key[R.groups]))
    assert info["count"].sum() == n and info["count"].max() <= G.MAX_ITEM
    perm = T.perm()
    assert np.array_equal(np.sort(perm), np.arange(n))


def test_batch_tree_is_concatenation_of_systems():
    systems = [W.plummer(n, seed=s) for s, n in ((1, 300), (2, 1000), (3, 17))]
    T = G.Tree.build_batch(systems, 8, 16)
    assert T.stats["n_sys"] == 3
    info = T.item_info()
    perm = T.perm()
    off = np.cumsum([0] + [len(m) for _, m in systems])
    for s, (pos, m) in enumerate(systems):
        R = O.Tree(pos, m, 8, 16)
        sel = info["sys"] == s
        assert np.array_equal(np.unique(info["group_key"][sel]), np.sort(R.key[R.groups]))
        assert info["count"][sel].sum() == len(m)
        seg = perm[off[s]:off[s + 1]]
        assert np.array_equal(np.sort(seg), np.arange(off[s], off[s + 1]))


def test_invalid_arguments_are_rejected_without_a_gpu():
    pos, m = W.plummer(100, seed=1)
    with pytest.raises(G.OctgravError) as e:
        G.Tree.build(pos, m, 0, 0)
    assert e.value.code == G.ERR_ARG
    with pytest.raises(G.OctgravError) as e:
        G.Tree.build(pos, m, 16, 8)
    assert e.value.code == G.ERR_ARG
    bad = pos.copy()
    bad[7, 1] = np.nan
    with pytest.raises(G.OctgravError) as e:
        G.Tree.build(bad, m, 16)
    assert e.value.code == G.ERR_NONFINITE
    neg = m.copy()
    neg[3] = -1.0
    with pytest.raises(G.OctgravError) as e:
        G.Tree.build(pos, neg, 16)
    assert e.value.code == G.ERR_NONFINITE
    for args in ((bad, m), (pos, neg)):  # the one-shot call checks the values in its first pass
        with pytest.raises(G.OctgravError) as e:
            G.forces(*args, 0.01, 0.5)
        assert e.value.code == G.ERR_NONFINITE
    inf = pos.copy()
    inf[99, 2] = np.inf
    with pytest.raises(G.OctgravError) as e:
        G.forces(inf, m, 0.01, 0.5)
    assert e.value.code == G.ERR_NONFINITE
    for eps, theta in ((0.0, 0.5), (-1.0, 0.5), (0.01, -0.1), (float("nan"), 0.5), (0.01, float("inf"))):
        with pytest.raises(G.OctgravError) as e:
            G.forces(pos, m, eps, theta)
        assert e.value.code == G.ERR_ARG
        T = G.Tree.build(pos, m, 16)
        with pytest.raises(G.OctgravError) as e:
            T.forces(eps, theta)
        assert e.value.code == G.ERR_ARG
    T = G.Tree.build(pos, m, 16)
    with pytest.raises(G.OctgravError) as e:
        T.set_launch(3)
    assert e.value.code == G.ERR_ARG
    assert T.status() == G.ERR_STATE          # no launch yet


def test_oneshot_phases_need_a_completed_call():
    with pytest.raises(G.OctgravError) as e:
        G.oneshot_phases()
    assert e.value.code == G.ERR_STATE


def test_item_split_for_large_groups():
    pos = np.zeros((150, 3))
    pos[:140] = [0.5, 0.5, 0.5]          # 140 coincident particles: one max-depth leaf
    pos[140:] = np.random.default_rng(3).random((10, 3))
    m = np.full(150, 1 / 150)
    T = G.Tree.build(pos, m, 4, 4)
    info = T.item_info()
    assert info["count"].max() <= 64 and info["count"].sum() == 150
    assert T.stats["max_group"] == 140
    T.set_launch(1)
    assert T.item_info()["count"].max() <= 32


def _expected_cuts(c, item_max, split):
    """Items of a group of c particles: full items, then the rest r whole or,
    with split at 64 per item, as 32 + (r - 32) when r is 33..48."""
    out = [item_max] * (c // item_max)
    r = c % item_max
    if r:
        out += [32, r - 32] if split and item_max == 64 and 32 < r <= 48 else [r]
    return out


def _check_item_cuts(T, item_max, split):
    info = T.item_info()
    keys, first, count = info["group_key"], info["first"], info["count"]
    starts = np.flatnonzero(np.r_[True, keys[1:] != keys[:-1]])
    ends = np.r_[starts[1:], len(keys)]
    n_cut = 0
    for a, b in zip(starts, ends):
        c = int(count[a:b].sum())
        assert list(count[a:b]) == _expected_cuts(c, item_max, split)
        assert np.array_equal(first[a:b], first[a] + np.r_[0, np.cumsum(count[a:b - 1])])
        n_cut += b - a > (c + item_max - 1) // item_max
    return n_cut


def test_items_follow_the_cutting_rule():
    """Two particles per lane: a 33..48-particle rest is cut into 32 + the
    rest; one particle per lane: items of 32 and the rest, nothing else."""
    pos, m = W.plummer(20000, seed=4)
    T = G.Tree.build(pos, m, 16, 128)
    n_cut = _check_item_cuts(T, 64, True)
    assert n_cut > 10  # the case occurs on this input
    assert T.stats["n_items"] == len(T.item_info()["count"])
    T.set_launch(1)
    assert _check_item_cuts(T, 32, True) == 0
    T.set_launch(2)
    assert _check_item_cuts(T, 64, True) == n_cut


def test_item_cut_at_the_rule_boundaries():
    """Nine clumps of coincident particles (each a leaf at the depth limit, and
    with N_leaf = N_group = 4 a group of its own) whose counts sit on both sides
    of every bound of the cutting rule (32, 48, 64 per item)."""
    counts = [32, 33, 48, 49, 56, 64, 65, 80, 81]
    rng = np.random.default_rng(8)
    centres = rng.random((len(counts), 3))
    pos = np.concatenate([np.tile(c, (k, 1)) for c, k in zip(centres, counts)])
    m = np.full(len(pos), 1.0 / len(pos))
    T = G.Tree.build(pos, m, 4, 4)
    assert T.stats["n_groups"] == len(counts)
    info = T.item_info()
    k = info["group_key"]
    starts = np.flatnonzero(np.r_[True, k[1:] != k[:-1]])
    ends = np.r_[starts[1:], len(k)]
    got = sorted(tuple(int(c) for c in info["count"][a:b]) for a, b in zip(starts, ends))
    want = sorted(tuple(_expected_cuts(c, 64, True)) for c in counts)
    assert got == want
    assert (32, 1) in got and (32, 16) in got and (49,) in got and (64, 1) in got and (64, 16) in got and (64, 17) in got


def test_host_builds_from_threads_agree():
    """Host builds started from four threads at once share the library's thread
    pool (one parallel region at a time) and give the single-thread tree: the
    same permutation, cell keys and FP64 cell properties."""
    import threading

    pos, m = W.plummer(120000, seed=71)
    ref = G.Tree.build(pos, m, 16, 64)
    ref_perm, ref_keys = ref.perm(), ref.cell_keys()
    ref_props = ref.cell_props()
    out, errors = [None] * 4, []

    def work(k):
        try:
            t = G.Tree.build(pos, m, 16, 64)
            out[k] = (t.perm(), t.cell_keys(), t.cell_props())
        except Exception as e:  # reported on the main thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for perm, keys, props in out:
        assert np.array_equal(perm, ref_perm) and np.array_equal(keys, ref_keys)
        for name in ref_props:
            assert np.array_equal(props[name], ref_props[name]), name


def test_criterion_file_round_trip(tmp_path):
    """A trained criterion saved with its tau and band loads back bit for bit."""
    rng = np.random.default_rng(4)
    rec = rng.standard_normal(G.MLP_RECORD).astype(np.float32)
    rec[12:24] = np.abs(rec[12:24]) + 0.1
    path = str(tmp_path / "crit.npz")
    G.save_criterion(path, rec, -3.25, 0.8, 1.3, 1.0, system="sphere+disc seed 6", groups=64)
    d = G.load_criterion(path)
    assert np.array_equal(d["record"].view(np.uint32), rec.view(np.uint32))
    assert (d["tau"], d["theta_lo"], d["theta_hi"], d["theta_fb"]) == (-3.25, 0.8, 1.3, 1.0)
    assert d["meta"] == {"system": "sphere+disc seed 6", "groups": "64"}
    np.savez(str(tmp_path / "other.npz"), record=rec)
    with pytest.raises(ValueError):
        G.load_criterion(str(tmp_path / "other.npz"))
    with pytest.raises(ValueError):
        G.save_criterion(path, rec[:100], -3.0, 0.8, 1.3, 1.0)
