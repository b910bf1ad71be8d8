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
    again = G.autotune(systems[:12], n_leaf=16, eps=0.01, theta=0.6, candidates=(16, 32, 64))
    assert again == best                                   # cached
    pos, m = systems[3]
    T = G.Tree.build(pos, m, 16, best["n_group"])
    T.set_launch(best["particles_per_lane"])
    acc, _ = T.forces(0.01, 0.6)
    ra, _, _, _, _ = O.Tree(pos, m, 16, best["n_group"]).forces(0.01, 0.6)
    assert O.rel_rms(acc, ra) <= TOL_RMS
