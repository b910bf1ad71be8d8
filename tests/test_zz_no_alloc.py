"""The allocation-free entry point (octgrav_forces_noalloc) against the
regular one (octgrav_forces_device).

Some callers cannot allocate device memory when they need forces: a
simulation whose own allocator owns every device byte, or a time-step loop
that cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
cause. They hand the library device memory they already own (the "arena" for
the tree arrays, here a torch tensor allocated up front) and the library keeps
its small scratch in a fixed array of its own. This file runs last so that a
failure here never hides another test's result.
"""
import ctypes as C

import numpy as np
import pytest

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


def _rel_rms(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_forces_device_on_two_calls(torch):
    pos, m = W.plummer(50000, seed=12)
    T = G.Tree.build(pos, m, 16, 64)
    ref = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    T.forces_device(0.01, 0.5, ref)
    torch.cuda.synchronize()
    assert T.status() == G.OK
    ref_h = ref.cpu().numpy().astype(np.float64)

    lib = G.load()
    need = C.c_size_t(0)
    assert lib.octgrav_forces_noalloc(T._h, None, C.byref(need), 1.0, 0.5, 1.0, None, None) == G.OK
    assert need.value > 0
    arena = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.full((T.n, 4), float("nan"), dtype=torch.float32, device="cuda")
        size = C.c_size_t(need.value)
        rc = lib.octgrav_forces_noalloc(T._h, C.c_void_p(arena.data_ptr()), C.byref(size), 0.01, 0.5, 1.0,
                                        C.c_void_p(out.data_ptr()), stream)
        assert rc == G.OK, lib.octgrav_last_error()
        got = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all(), call
        assert _rel_rms(got[:, :3], ref_h[:, :3]) <= 1e-5, call
        assert _rel_rms(got[:, 3], ref_h[:, 3]) <= 1e-5, call


def test_noalloc_rejects_small_arena_and_too_many_items(torch):
    pos, m = W.plummer(5000, seed=3)
    T = G.Tree.build(pos, m, 16, 64)
    need = T.noalloc_arena_bytes()
    arena = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(G.OctgravError) as e:
        T.forces_noalloc(0.01, 0.5, out, (arena.data_ptr(), need - 256))
    assert e.value.code == G.ERR_ARG
    # one particle per leaf and per group: more work items than the fixed scratch holds
    big_pos, big_m = W.uniform_cube(G.NOALLOC_MAX_ITEMS + 1000, seed=4)
    B = G.Tree.build(big_pos, big_m, 1, 1)
    assert B.stats["n_items"] > G.NOALLOC_MAX_ITEMS
    with pytest.raises(G.OctgravError) as e:
        B.forces_noalloc(0.01, 0.5, 0, (arena.data_ptr(), 1 << 40))
    assert e.value.code == G.ERR_ARG


def test_noalloc_with_a_gpu_built_tree(torch):
    pos, m = W.plummer(30000, seed=14)
    T = G.Tree.build_gpu(pos, m, 16, 64)
    ref = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    T.forces_device(0.01, 0.5, ref)
    torch.cuda.synchronize()
    arena = torch.empty(T.noalloc_arena_bytes(), dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(ref)
    T.forces_noalloc(0.01, 0.5, out, arena)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32))


def _random_record(seed):
    """A criterion record with a random network whose inputs are never out of range."""
    import oracle.mlp as M
    rec = np.zeros(48 + M.NPARAM, np.float32)
    rec[12:24] = 1.0                      # sigma
    rec[24:36] = -1e30                    # standardised-input range
    rec[36:48] = 1e30
    rec[48:] = M.init(seed).astype(np.float32)
    return rec


@pytest.mark.parametrize("gpu_built", [False, True])
def test_noalloc_applies_the_learned_criterion(torch, gpu_built):
    """A tree with the learned criterion is walked with it: the results equal
    octgrav_forces_device's bit for bit, on two calls in a row, and differ from
    the plain walk's."""
    pos, m = W.sphere_disc(40000, seed=6)
    T = (G.Tree.build_gpu if gpu_built else G.Tree.build)(pos, m, 16, 64)
    plain = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    T.forces_device(0.01, 0.5, plain)
    T.set_criterion(_random_record(3), tau=0.0, theta_lo=0.4, theta_hi=1.2, theta_fb=0.7)
    ref = torch.empty_like(plain)
    T.forces_device(0.01, 0.5, ref)
    torch.cuda.synchronize()
    assert T.status() == G.OK
    arena = torch.empty(T.noalloc_arena_bytes(), dtype=torch.uint8, device="cuda")
    ref_bits = ref.cpu().numpy().view(np.uint32)
    for call in range(2):
        out = torch.full_like(ref, float("nan"))
        T.forces_noalloc(0.01, 0.5, out, arena)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref_bits), call
    assert not np.array_equal(plain.cpu().numpy().view(np.uint32), ref_bits)


def test_noalloc_runs_a_split_tree_unsplit(torch):
    """A list split needs a per-part buffer, so the allocation-free call runs the
    tree unsplit: its result is the unsplit launch's, bit for bit."""
    pos, m = W.plummer(16384, seed=1)
    T = G.Tree.build(pos, m, 16, 64)
    ref = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    T.forces_device(0.01, 0.5, ref)
    T.set_split(4)
    arena = torch.empty(T.noalloc_arena_bytes(), dtype=torch.uint8, device="cuda")
    out = torch.full_like(ref, float("nan"))
    T.forces_noalloc(0.01, 0.5, out, arena)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32))
