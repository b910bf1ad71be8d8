"""Pair-by-pair parity of the learned opening criterion, and list parity of the
plain walk at the benchmark's configurations (Sec. 2.2, Listings 1-2).

Learned walk. The GPU captures, for chosen work items, its interaction lists
and every candidate that reached the network step (cell and FP32
prediction). From the lists the test rebuilds the (group, cell) pairs the walk
tested -- the children of the opened nodes, which are the root and every
proper ancestor of a list entry -- and the walk's decision on each. The FP64
oracle decides every pair with the same rule; its network is the tensor-core
reading of a 12 -> 64 -> 64 -> 1 network "with BF16 weights and FP32
accumulation": the record's weights rounded to BF16, the inputs and the first
hidden layer rounded to BF16 before they are multiplied, sums exact.
Required:

* the lists are a valid walk: each tested child lies in exactly one of cell
  list, leaf list (leaves only) and opened nodes (nodes only);
* every pair decided by the band (theta_hi opens, theta_lo accepts) or by the
  point-cell rule gets the oracle's decision: both sides evaluate the same
  FP32 tests, bit for bit;
* the candidates that reached the network are exactly the oracle's band pairs
  with h > 0, each tested once;
* on every candidate whose inputs both sides found in range,
  |y_gpu - y_oracle| <= delta, the per-pair bound derived below;
* the network's decision equals the oracle's wherever |y_oracle - tau| > delta,
  and the range decision wherever no input lies within its error bound of a
  range limit; pairs that fail either margin are counted as undecidable and
  must stay rare (< 0.5 %); the oracle's own walk with the same rule reaches
  the same lists wherever no pair was undecidable.

The bound delta (first order, per pair, in FP64 from the oracle's values).
Inputs: the GPU evaluates the 12 features in FP32 from FP32-rounded geometry
(unit roundoff e = 2^-24; coordinates of magnitude <= X); each box-to-cube gap
carries <= 8eX, so the distance d carries <= 14eX + 4ed; log2 by the hardware
approximation adds <= 2^-21 + 3 ulp of the result; a relative error r of its
argument adds r / ln 2. Standardisation (f - mu) * fl(1/sigma) adds
e(|f| + |mu|)/sigma + 3e|x|. This gives e_x per input. Rounding to BF16 is
monotone, so the GPU's BF16 input lies between the roundings of x - e_x and
x + e_x: where those agree it equals the oracle's exactly, elsewhere it
differs by at most the larger gap (one BF16 step). Network: z1 = W1 x + b1
then differs by |W1| dx + g13 (|W1||x| + |b1|), the BF16 hidden value again by
the straddle of relu(z1 -+ dz1), z2 = W2 h1 + b2 by |W2| dh1 + g65 (|W2||h1| +
|b2|), and y = w3 . relu(z2) + b3 by |w3| . dz2 + g66 (|w3| . |h2| + |b3|),
with g_n = 2 n e (FP32 accumulation of n terms, allowing the tensor cores'
own rounding twice the unit roundoff).

Plain walk at full size: the lists of sampled work items equal the oracle's as
key multisets at C2 (1M Plummer, N_group 512: groups split into items that
share the group's box, taken longest first), C3 (4M clustered, eps = 1e-3)
and C4 (256 systems in one tree).
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.mlp as M
from paper_1005_5384_gb300 import octgrav as G
from paper_1005_5384_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BAND = dict(theta_lo=0.8, theta_hi=1.3, theta_fb=1.0)
E32 = 2.0 ** -24   # FP32 unit roundoff
TAU = float(np.float32(-3.2))  # representable in FP32, as the kernel holds it


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()
    return t


@pytest.fixture(scope="module")
def record(torch):
    """The criterion as the benchmark trains it: C5's recipe on seed 6, 64 groups of N_group 256."""
    tpos, tm = W.sphere_disc(1 << 20, seed=6)
    TT = G.Tree.build(tpos, tm, 16, 256)
    groups = np.sort(np.random.default_rng(0).choice(TT.stats["n_groups"], 64, replace=False))
    f, lab, _ = TT.mlp_samples(groups, 0.35, 0.01)
    rec, _ = G.mlp_train(f, lab, steps=3000, batch=4096, lr=2e-3, seed=3)
    return np.asarray(rec, np.float32)


def _bf16(a):
    """Round FP32 values to BF16 (nearest, ties to even), returned as FP32."""
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def _oracle_net(rec):
    """The oracle's network for the record: W1, W2 rounded to BF16 as the GPU holds
    them; biases, output weights and the input scaling as stored (FP32)."""
    p = M.unpack(rec[48:].astype(np.float64))
    p["W1"] = _bf16(p["W1"]).astype(np.float64)
    p["W2"] = _bf16(p["W2"]).astype(np.float64)
    r = rec.astype(np.float64)
    net = dict(w=M.pack(p), mu=r[:12], sigma=r[12:24], fmin=r[24:36], fmax=r[36:48])
    return net, p


def _tested_pairs(R, kidx, cells, leaves):
    """The cells the walk tested (children of its opened nodes) and whether it
    opened each, rebuilt from one item's lists; checks that the lists are a walk."""
    ck = set(int(k) for k in cells)
    lk = set(int(k) for k in leaves)
    assert len(ck) == len(cells) and len(lk) == len(leaves), "a cell is listed twice"
    opened = {1}
    for k in list(ck) + list(lk):
        a = k >> 3
        while a >= 1 and a not in opened:
            opened.add(a)
            a >>= 3
    tested, gopen = [], []
    n_acc = n_leaf = 0
    for o in opened:
        co = kidx[o]
        assert not R.leaf[co], "an opened node is a leaf"
        for c in R.child[co]:
            if c < 0:
                continue
            kc = int(R.key[c])
            in_c, in_l, in_o = kc in ck, kc in lk, kc in opened
            assert in_c + in_l + in_o == 1, "a tested child is not classified exactly once"
            assert not in_l or R.leaf[c], "a node in the leaf list"
            assert not in_o or not R.leaf[c], "an opened leaf on the stack"
            n_acc += in_c
            n_leaf += in_l
            tested.append(int(c))
            gopen.append(not in_c)
    assert n_acc == len(ck) and n_leaf == len(lk), "a list entry is no child of an opened node"
    return np.array(tested, np.int64), np.array(gopen, bool)


def _input_error(R, gcell, cells, f, x, net):
    """Per pair and input: bound on |x_gpu - x_oracle| (module docstring)."""
    cu = R.cube[cells]
    h = cu[:, 3]
    l = 2.0 * h
    n = len(cells)
    fixed = np.concatenate([np.abs(R.bmin[gcell]), np.abs(R.bmax[gcell]), np.abs(R.cube[gcell, :3]),
                            np.abs(R.com[0])])  # the group's box and centre, the root's centre of mass
    per = np.concatenate([np.abs(cu[:, :3]) + h[:, None], np.abs(R.com[cells])], axis=1)
    X = np.maximum(per.max(axis=1), np.broadcast_to(fixed.max(), (n,)))
    d = 2.0 ** f[:, 1]
    dd = 14 * E32 * X + 4 * E32 * d

    def elog(v, dv):
        v = np.maximum(v, 1e-30)
        return dv / (v * math.log(2.0)) * 1.01 + 2.0 ** -21 + 3 * 2.0 ** -23 * np.abs(np.log2(v))
    ef = np.zeros_like(f)
    ef[:, 0] = elog(l, 2 * E32 * l)
    ef[:, 1] = elog(d, dd)
    r = 2.0 ** f[:, 2]
    ef[:, 2] = elog(r, 4 * E32 * r + 8 * E32 * E32 * X)
    ef[:, 3] = f[:, 3] * (dd / d + 3 * E32)
    M_ = 2.0 ** f[:, 4]
    ef[:, 4] = elog(M_, E32 * M_)
    ef[:, 5] = 12 * E32 * np.abs(f[:, 5])
    ef[:, 6] = elog(2.0 ** f[:, 6], 0.0)
    for k in (7, 8, 9):
        ef[:, k] = 3 * E32 * X / (2 * l) + 4 * E32 * np.abs(f[:, k])
    ef[:, 10] = 2 * E32 * np.abs(f[:, 10])
    o = 2.0 ** f[:, 11]
    ef[:, 11] = elog(o, 4 * E32 * o + 8 * E32 * E32 * X)
    return (ef + E32 * (np.abs(f) + np.abs(net["mu"]))) / net["sigma"] + 3 * E32 * np.abs(x)


def _straddle(lo, mid, hi):
    """Largest change of the BF16 rounding (by way of FP32) of any value in
    [lo, hi] from that of mid; 0 where the whole interval rounds alike."""
    r = _bf16(mid).astype(np.float64)
    return np.maximum(np.abs(_bf16(hi).astype(np.float64) - r), np.abs(r - _bf16(lo).astype(np.float64)))


def _network_bound(p, x, ex):
    """Per pair: bound on |y_gpu - y_oracle| given input errors ex, the oracle's
    network taking BF16 operands (module docstring)."""
    W1, b1, W2, b2, w3, b3 = p["W1"], p["b1"], p["W2"], p["b2"], p["w3"], p["b3"][0]
    A1, A2, a3 = np.abs(W1), np.abs(W2), np.abs(w3)
    xr = _bf16(x).astype(np.float64)
    dx = _straddle(x - ex, x, x + ex)
    z1 = xr @ W1.T + b1
    dz1 = dx @ A1.T + 2 * 13 * E32 * ((np.abs(xr) + dx) @ A1.T + np.abs(b1)) + 1e-12
    relu = lambda v: np.maximum(v, 0.0)  # noqa: E731
    hr = _bf16(relu(z1)).astype(np.float64)
    dh = _straddle(relu(z1 - dz1), relu(z1), relu(z1 + dz1))
    z2 = hr @ W2.T + b2
    dz2 = dh @ A2.T + 2 * 65 * E32 * ((hr + dh) @ A2.T + np.abs(b2)) + 1e-12
    return dz2 @ a3 + 2 * 66 * E32 * ((relu(z2) + dz2) @ a3 + abs(b3)) + 1e-12


def _check_learned_items(T, R, rec, theta_walk, items):
    """Run the capture on `items` and check every tested pair (module docstring).
    Returns (pairs, network pairs, undecidable pairs)."""
    net, p = _oracle_net(rec)
    caps = T.debug_walk(theta_walk, items=items, cap=8192, net_cap=16384)
    info = T.item_info()
    kidx = {int(k): c for c, k in enumerate(R.key)}
    gkey = {int(R.key[c]): g for g, c in enumerate(R.groups)}
    n_pairs = n_net = n_undec = n_edge = n_tau = 0
    net_in = dict(net, fmin=np.full(12, -np.inf), fmax=np.full(12, np.inf))
    net_out = dict(net, fmin=np.full(12, np.inf))
    decided = {}  # group -> (cell-list length, leaf-list particles) of items with no undecidable pair
    for it, cap in zip(items, caps):
        g = gkey[int(info["group_key"][it])]
        gcell = int(R.groups[g])
        tested, gopen = _tested_pairs(R, kidx, cap["cells"], cap["leaves"])
        op, br, y, f = R.mlp_decide_many(np.full(len(tested), g), tested, net, TAU, features=True, bf16=True,
                                         **BAND)
        n_pairs += len(tested)
        band = br <= 2
        assert np.array_equal(gopen[band], op[band]), ("band decision differs", it)
        # the network candidates: exactly the oracle's pairs in the band with h > 0
        nk = [kidx[int(k)] for k in cap["net_keys"]]
        assert len(set(nk)) == len(nk), ("a candidate reached the network twice", it)
        netpairs = tested[br >= 3]
        assert set(nk) == set(netpairs.tolist()), ("network candidates differ", it)
        sizes = (len(cap["cells"]), int(sum(R.count[kidx[int(k)]] for k in cap["leaves"])))
        if len(netpairs) == 0:
            decided[g] = sizes
            continue
        ygpu = dict(zip(nk, cap["net_y"].astype(np.float64)))
        sel = np.nonzero(br >= 3)[0]
        cs = tested[sel]
        gs = np.full(len(sel), g)
        # the oracle's two candidate outcomes of every band pair: the network's
        # (all inputs taken as in range) and the theta_fb fallback's
        op_net, _, y_net = R.mlp_decide_many(gs, cs, net_in, TAU, bf16=True, **BAND)
        op_fb, _, _ = R.mlp_decide_many(gs, cs, net_out, TAU, bf16=True, **BAND)
        fs = f[sel]
        x = (fs - net["mu"]) / net["sigma"]
        ex = _input_error(R, gcell, cs, fs, x, net)
        near_edge = np.any((np.abs(x - net["fmin"]) <= ex) | (np.abs(x - net["fmax"]) <= ex), axis=1)
        yg = np.array([ygpu[int(c)] for c in cs])
        g_in = ~np.isnan(yg)
        o_in = br[sel] == 4
        assert np.all((g_in == o_in) | near_edge), ("range decision differs away from a limit", it)
        delta = _network_bound(p, x, ex)
        err = np.abs(yg[g_in] - y_net[g_in])
        assert np.all(err <= delta[g_in]), ("prediction outside its bound", it, float(np.max(err - delta[g_in])))
        # the GPU followed its own prediction or the fallback test
        go = gopen[sel]
        assert np.array_equal(go[g_in], ~(yg[g_in] < TAU)), ("decision differs from own prediction", it)
        assert np.array_equal(go[~g_in], op_fb[~g_in]), ("fallback decision differs", it)
        # and took an outcome the oracle allows
        certain = np.abs(y_net - TAU) > delta
        net_ok = o_in | near_edge
        fb_ok = ~o_in | near_edge
        can_open = (net_ok & (op_net | ~certain)) | (fb_ok & op_fb)
        can_acc = (net_ok & (~op_net | ~certain)) | (fb_ok & ~op_fb)
        assert np.all(np.where(go, can_open, can_acc)), ("decision the oracle does not allow", it)
        undec = can_open & can_acc
        n_net += len(sel)
        n_undec += int(undec.sum())
        n_edge += int(near_edge.sum())
        n_tau += int((~certain).sum())
        if not undec.any():
            decided[g] = sizes
    print("network pairs %d: near a range limit %d, prediction within delta of tau %d, undecidable %d"
          % (n_net, n_edge, n_tau, n_undec))
    return n_pairs, n_net, n_undec, decided


def _oracle_walk_agrees(R, rec, decided):
    """The oracle's own walk with the same rule gives the same list sizes for
    every group whose pairs were all decidable (Listing 2 with the network)."""
    net, _ = _oracle_net(rec)
    groups = np.array(sorted(decided), np.int64)
    _, _, onpp, onpc, _ = R.forces_mlp(0.01, net, TAU, groups=groups, bf16=True, **BAND)
    for g in groups:
        i = int(R.cell_members(int(R.groups[g]))[0])
        assert (int(onpc[i]), int(onpp[i]) + 1) == decided[int(g)], int(g)
    return len(groups)


def test_learned_walk_decisions_pair_by_pair(torch, record):
    """A 131k sphere + disc (N_group 64): 400 sampled work items."""
    pos, m = W.sphere_disc(131072, seed=8)
    T = G.Tree.build(pos, m, 16, 64)
    T.set_criterion(record, tau=TAU, **BAND)
    R = O.Tree(pos, m, 16, 64)
    items = W.sample_indices(T.stats["n_items"], 400, seed=13)
    n_pairs, n_net, n_undec, decided = _check_learned_items(T, R, record, 0.5, items)
    print("pairs %d, network pairs %d, undecidable %d" % (n_pairs, n_net, n_undec))
    assert n_net > 0.05 * n_pairs
    assert n_undec <= 0.005 * n_net
    assert _oracle_walk_agrees(R, record, decided) >= 0.9 * len(items)


def test_learned_walk_decisions_at_benchmark_scale(torch, record):
    """C5 as the benchmark runs it (1M sphere + disc, N_group 256, items longest
    first): 200 sampled work items plus the largest one."""
    pos, m = W.sphere_disc(1 << 20, seed=5)
    T = G.Tree.build(pos, m, 16, 256)
    T.set_criterion(record, tau=TAU, **BAND)
    out = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    T.forces_device(0.01, 0.5, out)
    T.balance()
    R = O.Tree(pos, m, 16, 256)
    info = T.item_info()
    items = np.union1d(W.sample_indices(T.stats["n_items"], 200, seed=14), [int(np.argmax(info["count"]))])
    n_pairs, n_net, n_undec, decided = _check_learned_items(T, R, record, 0.5, items)
    print("pairs %d, network pairs %d, undecidable %d" % (n_pairs, n_net, n_undec))
    assert n_net > 0.05 * n_pairs
    assert n_undec <= 0.005 * n_net
    assert _oracle_walk_agrees(R, record, decided) >= 0.8 * len(set(int(g) for g in info["group_key"][items]))


# ---------------------------------------------------------------- plain walk: full-size list parity

def _list_parity(T, Rs, theta, items, sys_of_item=None):
    """Lists of `items` equal the oracle's (per-system oracle trees Rs) as key multisets."""
    caps = T.debug_walk(theta, items=items, cap=16384)
    info = T.item_info()
    gkeys = [None if R is None else {int(R.key[c]): g for g, c in enumerate(R.groups)} for R in Rs]
    for it, cap in zip(items, caps):
        s = int(info["sys"][it]) if sys_of_item else 0
        R = Rs[s]
        g = gkeys[s][int(info["group_key"][it])]
        oc, ol = R.list_keys(g, theta)
        assert np.array_equal(cap["cells"], oc), ("cell list", it)
        assert np.array_equal(cap["leaves"], ol), ("leaf list", it)


def _sample_items(T, k, seed):
    info = T.item_info()
    big = np.argsort(info["count"])[-3:]
    return np.union1d(W.sample_indices(T.stats["n_items"], k, seed=seed), big)


def test_list_parity_plummer_1m_n_group_512(torch):
    """C2 at the benchmark's configuration: groups of up to 512 particles split
    into work items that share the group's box, items taken longest first."""
    pos, m = W.plummer(1 << 20, seed=1)
    T = G.Tree.build(pos, m, 16, 512)
    out = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    T.forces_device(0.01, 0.5, out)
    T.balance()
    items = _sample_items(T, 300, 21)
    info = T.item_info()
    assert np.any(info["count"][items] < 64) and len(np.unique(info["group_key"])) < T.stats["n_items"]
    _list_parity(T, [O.Tree(pos, m, 16, 512)], 0.5, items)


def test_list_parity_plummer_1m_n_group_256_cut_items(torch):
    """C2 as the benchmark runs it now (the autotuner's N_group 256, items
    longest first): a group's 33..48-particle rest is cut into 32 + the rest,
    and both pieces walk the group's lists. The sample holds both pieces of
    20 cut groups besides 300 random items."""
    pos, m = W.plummer(1 << 20, seed=1)
    T = G.Tree.build(pos, m, 16, 256)
    out = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    T.forces_device(0.01, 0.5, out)
    T.balance()
    info = T.item_info()
    k, cnt = info["group_key"], info["count"]
    starts = np.flatnonzero(np.r_[True, k[1:] != k[:-1]])
    ends = np.r_[starts[1:], len(k)]
    cut = [(a, b) for a, b in zip(starts, ends)
           if b - a >= 2 and cnt[b - 2] == 32 and 1 <= cnt[b - 1] <= 16 and int(cnt[a:b].sum()) % 64 != 0]
    assert len(cut) > 100
    pick = np.random.default_rng(5).choice(len(cut), 20, replace=False)
    pieces = [i for j in pick for i in (cut[j][1] - 2, cut[j][1] - 1)]
    items = np.union1d(_sample_items(T, 300, 24), pieces)
    _list_parity(T, [O.Tree(pos, m, 16, 256)], 0.5, items)


def test_list_parity_clustered_4m(torch):
    """C3: 64 Plummer spheres, 4M particles, eps = 1e-3 (lists do not depend on eps)."""
    pos, m = W.clustered()
    T = G.Tree.build(pos, m, 16, 256)
    _list_parity(T, [O.Tree(pos, m, 16, 256)], 0.5, _sample_items(T, 300, 22))


def test_list_parity_ensemble_batch(torch):
    """C4: 256 independent systems in one tree, theta = 0.6; items of every size class."""
    systems = W.ensemble()
    T = G.Tree.build_batch(systems, 16, 256)
    items = _sample_items(T, 300, 23)
    info = T.item_info()
    need = sorted(set(int(s) for s in info["sys"][items]))
    Rs = [None] * len(systems)
    for s in need:
        Rs[s] = O.Tree(systems[s][0], systems[s][1], 16, 256)
    _list_parity(T, Rs, 0.6, items, sys_of_item=True)


def test_debug_walk_subset_equals_full_capture_and_refusals(torch):
    """A capture of chosen work items returns exactly the rows of a full capture;
    bad item lists are refused and the tree stays usable."""
    pos, m = W.plummer(20000, seed=4)
    T = G.Tree.build(pos, m, 16, 64)
    full = T.debug_walk(0.5, cap=4096)
    sel = np.array([7, 0, T.stats["n_items"] - 1, 123])
    part = T.debug_walk(0.5, items=sel, cap=4096)
    for r, it in enumerate(sel):
        assert np.array_equal(part[r]["cells"], full[it]["cells"])
        assert np.array_equal(part[r]["leaves"], full[it]["leaves"])
    for bad in ([0, 0], [-1], [T.stats["n_items"]]):
        with pytest.raises(G.OctgravError) as e:
            T.debug_walk(0.5, items=np.array(bad), cap=4096)
        assert e.value.code == G.ERR_ARG
    with pytest.raises(G.OctgravError) as e:
        T.debug_walk(0.5, items=sel, cap=2)  # lists longer than the capture buffer
    assert e.value.code == G.ERR_LIST
    assert T.debug_walk(0.5, items=sel[:1], cap=4096)[0]["cells"].size == full[7]["cells"].size
    assert T.debug_walk(0.5, items=np.array([], np.int64), cap=16) == []
