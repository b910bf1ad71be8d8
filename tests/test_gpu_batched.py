"""Batched ensembles (many independent systems in one persistent launch), CUDA
graph capture/replay and the autotuner, checked against the FP64 oracle run
system by system."""
import numpy as np
import pytest

import oracle as O
from paper_1005_5384_gb300 import octgrav as G
from paper_1005_5384_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL_RMS = 1e-5


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()
    return t


@pytest.fixture(scope="module")
def systems():
    return W.ensemble(24, seed=4, n_min=200, n_max=6000)


def test_batched_forces_match_per_system_oracle(torch, systems):
    rng = np.random.default_rng(2)
    eps = 0.005 + 0.015 * rng.random(len(systems))
    theta = 0.4 + 0.4 * rng.random(len(systems))
    T = G.Tree.build_batch(systems, 16, 32)
    T.set_system_params(eps, theta)
    acc, pot = T.forces(1.0, 1.0)          # scalar eps/theta are overridden per system
    off = T.offsets
    for s, (pos, m) in enumerate(systems):
        R = O.Tree(pos, m, 16, 32)
        ra, rp, _, _, _ = R.forces(eps[s], theta[s])
        a, p = acc[off[s]:off[s + 1]], pot[off[s]:off[s + 1]]
        assert O.rel_rms(a, ra) <= TOL_RMS, s
        assert float(np.linalg.norm(p - rp) / np.linalg.norm(rp)) <= TOL_RMS, s


def test_batched_lists_bit_exact(torch, systems):
    sub = systems[:8]
    T = G.Tree.build_batch(sub, 16, 32)
    lists = T.debug_lists(0.6, cap=4096)
    info = T.item_info()
    oracles = [O.Tree(p, m, 16, 32) for p, m in sub]
    okeys = [{int(R.key[c]): g for g, c in enumerate(R.groups)} for R in oracles]
    for k, (ck, lk) in enumerate(lists):
        s = int(info["sys"][k])
        R = oracles[s]
        rc, rl = R.list_keys(okeys[s][int(info["group_key"][k])], 0.6)
        assert np.array_equal(ck, rc) and np.array_equal(lk, rl), (k, s)


def test_graph_replay_equals_direct_launch(torch, systems):
    T = G.Tree.build_batch(systems, 16, 64)
    out1 = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    T.forces_device(0.01, 0.6, out1)
    torch.cuda.synchronize()
    ref = out1.cpu().numpy().copy()
    c_ref = T.interaction_counts()
    stream = torch.cuda.Stream()
    out2 = torch.full((T.n, 4), float("nan"), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        T.capture_graph(0.01, 0.6, out2, stream=stream)
        for _ in range(2):
            T.launch_graph(stream=stream)
    stream.synchronize()
    assert T.status(stream=stream) == G.OK
    assert np.array_equal(out2.cpu().numpy(), ref)
    assert T.interaction_counts(stream=stream) == c_ref


def test_autotuner_returns_a_valid_configuration(torch, systems):
    best = G.autotune(systems[:12], n_leaf=16, eps=0.01, theta=0.6, candidates=(16, 32, 64))
    assert best["n_group"] in (16, 32, 64) and best["particles_per_lane"] in (1, 2) and best["ms"] > 0
    assert best["split"] in (1, 2, 4) and best["staging"] in (0, 1, 2)
    assert best["split"] == 1 or best["staging"] == 1      # a split runs with cp.async staging
    again = G.autotune(systems[:12], n_leaf=16, eps=0.01, theta=0.6, candidates=(16, 32, 64))
    assert again == best                                   # cached
    plain = G.autotune(systems[:12], n_leaf=16, eps=0.01, theta=0.6, candidates=(16, 32, 64), staging=False)
    assert plain["staging"] == 1 and plain["n_group"] in (16, 32, 64)
    pos, m = systems[3]
    T = G.Tree.build(pos, m, 16, best["n_group"])
    T.set_launch(best["particles_per_lane"])
    T.set_staging(best["staging"])
    acc, _ = T.forces(0.01, 0.6)
    ra, _, _, _, _ = O.Tree(pos, m, 16, best["n_group"]).forces(0.01, 0.6)
    assert O.rel_rms(acc, ra) <= TOL_RMS


def test_autotuner_ex_writes_at_most_n_best_values(torch, systems):
    """octgrav_autotune_ex fills min(n_best, 4) values and refuses n_best < 1."""
    import ctypes as C
    lib = G.load()
    sub = systems[:4]
    pos = np.ascontiguousarray(np.concatenate([p for p, _ in sub]))
    mass = np.ascontiguousarray(np.concatenate([m for _, m in sub]))
    off = np.zeros(len(sub) + 1, np.int64)
    off[1:] = np.cumsum([len(m) for _, m in sub])
    cand = np.array([16, 32], np.int32)
    best = np.full(6, -7, np.int32)
    ms = np.zeros(1)
    rc = lib.octgrav_autotune_ex(len(sub), off, pos.reshape(-1), mass, 16, 0.01, 0.6, cand.ctypes.data, 2,
                                 best.ctypes.data, 2, ms.ctypes.data, None)
    assert rc == G.OK, lib.octgrav_last_error()
    assert best[0] in (16, 32) and best[1] in (1, 2) and np.all(best[2:] == -7) and ms[0] > 0
    rc = lib.octgrav_autotune_ex(len(sub), off, pos.reshape(-1), mass, 16, 0.01, 0.6, cand.ctypes.data, 2,
                                 best.ctypes.data, 0, ms.ctypes.data, None)
    assert rc == G.ERR_ARG


def test_autotuner_cache_tells_distributions_apart(torch):
    """Same size, theta, eps and N_leaf but a different spread (Plummer sphere vs
    uniform cube): the second call is tuned, not served from the cache."""
    import time
    a = W.plummer(20000, seed=31)
    b = W.uniform_cube(20000, seed=31)
    G.autotune([a], n_leaf=16, eps=0.01, theta=0.55, candidates=(32, 64))
    t0 = time.perf_counter()
    G.autotune([a], n_leaf=16, eps=0.01, theta=0.55, candidates=(32, 64))
    cached = time.perf_counter() - t0
    t0 = time.perf_counter()
    G.autotune([b], n_leaf=16, eps=0.01, theta=0.55, candidates=(32, 64))
    tuned = time.perf_counter() - t0
    assert tuned > 5 * cached


def test_one_shot_batched_call_matches_per_system_oracle(torch, systems):
    """octgrav_forces_batched: host arrays and per-system eps / theta in, FP64
    results in input order out; each system equals the oracle run on it alone,
    and the whole equals the three-call path (batch build, per-system
    parameters, forces) bit for bit."""
    rng = np.random.default_rng(7)
    eps = 0.005 + 0.015 * rng.random(len(systems))
    theta = 0.4 + 0.4 * rng.random(len(systems))
    acc, pot = G.forces_batched(systems, eps, theta, n_group=64)
    off = np.zeros(len(systems) + 1, np.int64)
    off[1:] = np.cumsum([len(m) for _, m in systems])
    for s, (pos, m) in enumerate(systems):
        ra, rp, _, _, _ = O.Tree(pos, m, 16, 64).forces(eps[s], theta[s])
        a, p = acc[off[s]:off[s + 1]], pot[off[s]:off[s + 1]]
        assert O.rel_rms(a, ra) <= TOL_RMS, s
        assert float(np.linalg.norm(p - rp) / np.linalg.norm(rp)) <= TOL_RMS, s
    T = G.Tree.build_batch(systems, 16, 64)
    T.set_system_params(eps, theta)
    a3, p3 = T.forces(1.0, 1.0)
    assert np.array_equal(acc, a3) and np.array_equal(pot, p3)
    # the defaults (N_leaf 16, N_group 256, G = 1) through the plain entry point
    lib = G.load()
    pos = np.ascontiguousarray(np.concatenate([p for p, _ in systems]))
    mass = np.ascontiguousarray(np.concatenate([m for _, m in systems]))
    a0 = np.empty_like(acc)
    p0 = np.empty_like(pot)
    rc = lib.octgrav_forces_batched(len(systems), off, pos.ctypes.data_as(G._vp), mass.ctypes.data_as(G._vp),
                                    eps, theta, a0.ctypes.data_as(G._vp), p0.ctypes.data_as(G._vp), None)
    assert rc == G.OK, lib.octgrav_last_error()
    a1, p1 = G.forces_batched(systems, eps, theta, n_group=256)
    assert np.array_equal(a0, a1) and np.array_equal(p0, p1)


def test_one_shot_batched_call_refusals(torch, systems):
    sub = systems[:3]
    with pytest.raises(G.OctgravError) as e:
        G.forces_batched(sub, [0.01, -1.0, 0.01], 0.5)
    assert e.value.code == G.ERR_ARG
    with pytest.raises(G.OctgravError) as e:
        G.forces_batched(sub, 0.01, [0.5, np.nan, 0.5])
    assert e.value.code == G.ERR_ARG
    bad = [(p.copy(), m.copy()) for p, m in sub]
    bad[1][0][5, 2] = np.inf
    with pytest.raises(G.OctgravError) as e:
        G.forces_batched(bad, 0.01, 0.5)
    assert e.value.code == G.ERR_NONFINITE
    pos = np.concatenate([p for p, _ in sub])
    mass = np.concatenate([m for _, m in sub])
    with pytest.raises(G.OctgravError) as e:
        G.forces_batched((np.array([0, 5, 5, len(mass)]), pos, mass), 0.01, 0.5)
    assert e.value.code == G.ERR_ARG
    # the context stays usable
    acc, _ = G.forces_batched(sub, 0.01, 0.5)
    assert np.isfinite(acc).all()
