"""Learned opening criterion on the GPU against the FP64 oracle.

* the training kernels' gradient equals the oracle network's FP64 backward pass;
* the GPU-made training samples (features, FP64 error labels) equal the
  oracle's for the same (group, cell) pairs;
* the trained network predicts held-out labels;
* a walk with the learned criterion: its forces equal the oracle's evaluation
  of the same lists within 1e-5 (its decisions are checked pair by pair in
  test_gpu_decisions.py);
* the gain: at an equal median relative force error of 1e-3 the learned walk
  needs fewer interactions and less time than the plain theta walk.
"""

import numpy as np
import pytest

import oracle as O
import oracle.mlp as M
from paper_1005_5384_gb300 import octgrav as G
from paper_1005_5384_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BAND = dict(theta_lo=0.8, theta_hi=1.3, theta_fb=1.0)


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()
    return t


@pytest.fixture(scope="module")
def trained(torch):
    pos, m = W.sphere_disc(131072, seed=6)
    T = G.Tree.build(pos, m, 16, 64)
    groups = np.sort(np.random.default_rng(0).choice(T.stats["n_groups"], 48, replace=False))
    f, lab, pairs = T.mlp_samples(groups, 0.35, 0.01)
    rec, loss = G.mlp_train(f, lab, steps=2000, batch=4096, lr=2e-3, seed=3)
    return dict(pos=pos, m=m, T=T, groups=groups, f=f, lab=lab, pairs=pairs, rec=rec, loss=loss)


def _net(rec):
    rec = np.asarray(rec, np.float64)
    return dict(mu=rec[:12], sigma=rec[12:24], fmin=rec[24:36], fmax=rec[36:48], w=rec[48:])


def test_gpu_gradient_matches_oracle_backward(torch):
    rng = np.random.default_rng(11)
    w = (M.init(5) + 0.05 * rng.standard_normal(M.NPARAM)).astype(np.float32)
    X = rng.standard_normal((300, 12)).astype(np.float32)
    t = (rng.standard_normal(300) * 2).astype(np.float32)
    g_gpu, L_gpu = G.mlp_grad(w, X, t)
    L, g = M.loss_and_grad(w.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert L_gpu == pytest.approx(L, rel=1e-5)
    assert np.abs(g_gpu - g).max() <= 1e-4 * np.abs(g).max()


def test_gpu_samples_match_oracle(trained):
    T, pos, m = trained["T"], trained["pos"], trained["m"]
    R = O.Tree(pos, m, 16, 64)
    aref, _, _, _, _ = R.forces(0.01, 0.3, counts=False)
    of, olab, opairs = R.mlp_samples(trained["groups"], 0.35, 0.01, aref)
    keys = T.cell_keys()
    gpu = {(int(g), int(keys[c])): k for k, (g, c) in enumerate(trained["pairs"])}
    ora = {(int(g), int(R.key[c])): k for k, (g, c) in enumerate(opairs)}
    # both sides take a pair when the FP32 test sees h > 0 and a nonzero gap
    assert len(gpu) == len(trained["pairs"]) and len(ora) == len(opairs)
    assert set(gpu) == set(ora)
    common = set(gpu)
    gi = np.array([gpu[k] for k in common])
    oi = np.array([ora[k] for k in common])
    fg, fo = trained["f"][gi].astype(np.float64), of[oi]
    # distances (features 1, 2, 11 are their log2) come from FP32 coordinates of
    # order 1: compare them linearly to an absolute FP32-scale tolerance
    for k in (1, 2, 11):
        assert np.all(np.abs(2.0 ** fg[:, k] - 2.0 ** fo[:, k]) <= 2e-6), k
    far = 2.0 ** fo[:, 1] > 1e-3
    assert np.all(np.abs(fg[far, 3] - fo[far, 3]) <= 1e-4 * fo[far, 3])
    for k in (0, 4, 5, 6, 7, 8, 9, 10):
        assert np.all(np.abs(fg[:, k] - fo[:, k]) <= 1e-4 * (1.0 + np.abs(fo[:, k]))), k
    lg, lo = trained["lab"][gi].astype(np.float64), olab[oi]
    big = lo > 1e-9
    assert np.all(np.abs(lg[big] - lo[big]) <= 1e-3 * lo[big])


def test_training_learns_the_labels(trained):
    y = np.log10(np.maximum(trained["lab"].astype(np.float64), 1e-12))
    assert trained["loss"] < 0.25 * 0.5 * y.var()
    # held-out groups of the same system
    T = trained["T"]
    rest = np.setdiff1d(np.arange(T.stats["n_groups"]), trained["groups"])
    hold = np.sort(np.random.default_rng(9).choice(rest, 12, replace=False))
    f, lab, _ = T.mlp_samples(hold, 0.35, 0.01)
    net = _net(trained["rec"])
    X = (f.astype(np.float64) - net["mu"]) / net["sigma"]
    pred, _ = M.forward(net["w"], X)
    rmse = np.sqrt(np.mean((pred - np.log10(np.maximum(lab.astype(np.float64), 1e-12))) ** 2))
    assert rmse < 0.6, rmse


def test_learned_walk_forces_on_its_lists(torch, trained):
    pos, m = W.sphere_disc(32768, seed=8)
    T = G.Tree.build(pos, m, 16, 64)
    tau = -3.5
    T.set_criterion(trained["rec"], tau=tau, **BAND)
    acc, pot = T.forces(0.01, 0.5)
    lists = T.debug_lists(0.5, cap=8192)
    info = T.item_info()
    R = O.Tree(pos, m, 16, 64)
    kidx = {int(k): c for c, k in enumerate(R.key)}
    okey = {int(R.key[c]): g for g, c in enumerate(R.groups)}
    num = den = 0.0
    seen = set()
    for k, (ck, lk) in enumerate(lists):
        g = okey[int(info["group_key"][k])]
        if g in seen:
            continue
        seen.add(g)
        ra, rp = R.forces_on_lists(g, [kidx[int(v)] for v in ck], [kidx[int(v)] for v in lk], 0.01)
        mem = R.cell_members(int(R.groups[g]))
        num += float(np.sum((acc[mem] - ra) ** 2))
        den += float(np.sum(ra ** 2))
    assert np.sqrt(num / den) <= 1e-5


def _median_err(T, torch, out, eps, samp, ad, theta):
    T.forces_device(eps, theta, out)
    torch.cuda.synchronize()
    acc = np.empty((T.n, 3))
    acc[T.perm()] = out.cpu().numpy()[:, :3]
    return float(np.median(O.rel_err(acc[samp], ad)))


def _bisect(f, lo, hi, target=1e-3, iters=10, increasing=True):
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if (f(mid) < target) == increasing:
            lo = mid
        else:
            hi = mid
    return lo


def _time_events(T, torch, out, eps, theta, reps=9):
    """Median launch time (ms) between CUDA events on the current stream."""
    T.forces_device(eps, theta, out)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        T.forces_device(eps, theta, out)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def test_learned_criterion_beats_theta_at_equal_median_error(torch):
    """C5 as the benchmark runs it: the network trained on another seed of the
    same kind of system (256 groups; their samples with cell size over distance
    at least 0.7 theta_lo), N_group 256; the plain walk and the learned
    walk each tuned to a median Delta a/a of 1e-3 against FP64 direct sums at
    1024 particles; both timed with CUDA events after ordering their items
    longest first. The learned walk needs at least 20 % fewer flops and runs
    at least 5 % faster (measured: ~38 % and ~16-20 %)."""
    tpos, tm = W.sphere_disc(1 << 20, seed=6)
    TT = G.Tree.build(tpos, tm, 16, 256)
    groups = np.sort(np.random.default_rng(0).choice(TT.stats["n_groups"], 256, replace=False))
    f, lab, _ = TT.mlp_samples(groups, 0.35, 0.01)
    keep = f[:, 3] >= 0.7 * BAND["theta_lo"]  # pairs the plain test accepts never reach the network
    rec, _ = G.mlp_train(np.ascontiguousarray(f[keep]), np.ascontiguousarray(lab[keep]), steps=3000, batch=4096,
                         lr=2e-3, seed=3)
    del TT
    pos, m = W.sphere_disc(1 << 20, seed=5)
    T = G.Tree.build(pos, m, 16, 256)
    out = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    samp = W.sample_indices(T.n, 1024, seed=23)
    ad, _ = O.direct(pos, m, 0.01, targets=samp)  # the error reference: FP64 direct sums of the oracle
    th = _bisect(lambda x: _median_err(T, torch, out, 0.01, samp, ad, x), 0.3, 2.0, iters=14)
    e_th = _median_err(T, torch, out, 0.01, samp, ad, th)
    f_th = T.interaction_counts()["flops"]
    T.balance()
    t_th = _time_events(T, torch, out, 0.01, th)
    T.balance(0)

    def err_tau(tau):
        T.set_criterion(rec, tau=tau, **BAND)
        return _median_err(T, torch, out, 0.01, samp, ad, 0.5)
    tau = _bisect(err_tau, -6.0, -1.0, iters=14)
    e_ml = err_tau(tau)
    f_ml = T.interaction_counts()["flops"]
    T.balance()
    t_ml = _time_events(T, torch, out, 0.01, 0.5)
    print("theta %.3f err %.2e flops %.3g time %.3f ms | tau %.3f err %.2e flops %.3g time %.3f ms"
          % (th, e_th, f_th, t_th, tau, e_ml, f_ml, t_ml))
    # the comparison is at equal error: both bisections end just below 1e-3
    # (14 halvings; the median error moves in small steps with the opening decisions)
    assert 0.93e-3 <= e_th <= 1.0e-3 and 0.93e-3 <= e_ml <= 1.0e-3
    assert abs(e_ml - e_th) <= 0.07 * e_th
    assert f_ml < 0.8 * f_th
    assert t_ml < 0.95 * t_th
