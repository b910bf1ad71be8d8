"""CPU FP64 oracle of the grouped Barnes-Hut force calculation (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package. It shares no code with the CUDA path: the arithmetic
lives in ``octgrav_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module compiles it on demand and marshals numpy
arrays through ctypes.

Steps (Gaburov, Bedorf & Portegies Zwart 2010):
  direct()        O1  direct Plummer-softened summation (Sec. 3.1 reference)
  Tree(...)       O2/O3 octree, tight boxes, boundary cubes, moments, groups
                  (Sec. 2.1, Fig. 1)
  open_f32()      O4  opening test (Sec. 2.2, Listing 2)
  Tree.lists()    O5  walk + list classification (Sec. 2.2, Listings 1-2)
  Tree.forces()   O6  particle-cell (monopole + quadrupole) and particle-leaf
                  evaluation (Sec. 2.3, Listings 3-4)
  Tree.mlp_*      O8  learned opening criterion: features, error labels, the
                  walk that consults the network (see oracle/mlp.py)
  leapfrog()      O9  kick-drift-kick time integration with direct forces
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "octgrav_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboctgrav_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_DEPTH = 21

_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboctgrav_oracle.so (gcc, -O2)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        lib.ora_direct.argtypes = [_f64p, _f64p, C.c_int64, C.c_void_p, C.c_int64, C.c_double,
                                   C.c_double, _f64p, _f64p, C.c_int]
        lib.ora_direct.restype = C.c_int
        lib.ora_tree_build.argtypes = [_f64p, _f64p, C.c_int64, C.c_int, C.c_int, C.c_int]
        lib.ora_tree_build.restype = C.c_void_p
        lib.ora_tree_free.argtypes = [C.c_void_p]
        lib.ora_tree_free.restype = None
        lib.ora_tree_info.argtypes = [C.c_void_p, _i64p]
        lib.ora_tree_frame.argtypes = [C.c_void_p, _f64p]
        lib.ora_tree_cells.argtypes = [C.c_void_p] + [C.c_void_p] * 13
        lib.ora_tree_members.argtypes = [C.c_void_p, _i64p]
        lib.ora_tree_groups.argtypes = [C.c_void_p, _i64p]
        lib.ora_walk.argtypes = [C.c_void_p, C.c_int64, C.c_double, _i64p, C.c_int64, _i64p,
                                 _i64p, C.c_int64, _i64p]
        lib.ora_walk.restype = C.c_int64
        lib.ora_forces.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_void_p,
                                   C.c_int64, _f64p, _f64p, C.c_void_p, C.c_void_p, C.c_int]
        lib.ora_forces.restype = C.c_int64
        lib.ora_open_f32.argtypes = [_f32p, _f32p, _f32p, C.c_float, C.c_float]
        lib.ora_open_f32.restype = C.c_int
        lib.ora_cell_field.argtypes = [_f64p, C.c_double, _f64p, _f64p, C.c_double, C.c_double,
                                       _f64p, _f64p]
        lib.ora_cell_field.restype = None
        lib.ora_mlp_features.argtypes = [C.c_void_p, C.c_int64, C.c_int64, _f64p]
        lib.ora_mlp_features.restype = None
        lib.ora_mlp_samples.argtypes = [C.c_void_p, _i64p, C.c_int64, C.c_double, C.c_double, _f64p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int]
        lib.ora_mlp_samples.restype = C.c_int64
        lib.ora_mlp_forward.argtypes = [_f64p, _f64p]
        lib.ora_mlp_forward.restype = C.c_double
        lib.ora_mlp_forward_bf16.argtypes = [_f64p, _f64p]
        lib.ora_mlp_forward_bf16.restype = C.c_double
        lib.ora_forces_mlp.argtypes = [C.c_void_p, C.c_double, C.c_double, _f64p, _f64p, _f64p, _f64p, _f64p,
                                       C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_void_p,
                                       C.c_int64, _f64p, _f64p, C.c_void_p, C.c_void_p, C.c_int]
        lib.ora_forces_mlp.restype = C.c_int64
        lib.ora_forces_on_lists.argtypes = [C.c_void_p, C.c_int64, _i64p, C.c_int64, _i64p, C.c_int64,
                                            C.c_double, C.c_double, _f64p, _f64p]
        lib.ora_forces_on_lists.restype = None
        lib.ora_mlp_decide.argtypes = [C.c_void_p, C.c_int64, C.c_int64, _f64p, _f64p, _f64p, _f64p, _f64p,
                                       C.c_double, C.c_double, C.c_double, C.c_double, C.c_int,
                                       C.POINTER(C.c_int), C.POINTER(C.c_double)]
        lib.ora_mlp_decide.restype = C.c_int
        lib.ora_mlp_decide_many.argtypes = [C.c_void_p, C.c_int64, _i64p, _i64p, _f64p, _f64p, _f64p, _f64p,
                                            _f64p, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int,
                                            _i32p, _i32p, _f64p, C.c_void_p]
        lib.ora_mlp_decide_many.restype = C.c_int
        _lib = lib
        return lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def direct(pos, mass, eps: float, G: float = 1.0, targets=None, nthreads: int | None = None):
    """O1: (acc [nt,3], pot [nt]) at ``targets`` (all particles when None)."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    n = mass.shape[0]
    if targets is None:
        nt, tp, tarr = n, None, None
    else:
        tarr = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp = tarr.shape[0], tarr.ctypes.data_as(C.c_void_p)
    acc = np.zeros((nt, 3))
    pot = np.zeros(nt)
    lib.ora_direct(pos.reshape(-1), mass, n, tp, nt, float(eps), float(G), acc.reshape(-1), pot,
                   int(nthreads or default_threads()))
    return acc, pot


def leapfrog(pos, vel, mass, eps: float, dt: float, n_steps: int, G: float = 1.0, nthreads: int | None = None):
    """O9: kick-drift-kick leapfrog with one shared step and direct-sum forces (O1).

    The paper integrates on the host and does not name its scheme; this is
    the standard second-order symplectic one. Per step: v += a dt/2,
    x += v dt, a = forces(x), v += a dt/2. Returns (pos, vel, acc, pot).
    """
    x = np.array(pos, dtype=np.float64, copy=True)
    v = np.array(vel, dtype=np.float64, copy=True)
    m = np.ascontiguousarray(mass, dtype=np.float64)
    a, phi = direct(x, m, eps, G, nthreads=nthreads)
    h = 0.5 * dt
    for _ in range(int(n_steps)):
        v = v + a * h
        x = x + v * dt
        a, phi = direct(x, m, eps, G, nthreads=nthreads)
        v = v + a * h
    return x, v, a, phi


def energies(vel, mass, pot):
    """(kinetic, potential) = (sum m v^2 / 2, sum m phi / 2) in FP64."""
    v = np.asarray(vel, dtype=np.float64)
    m = np.asarray(mass, dtype=np.float64)
    return 0.5 * float(np.sum(m * np.einsum("ij,ij->i", v, v))), 0.5 * float(np.sum(m * np.asarray(pot)))


def theta2_f32(theta: float) -> np.float32:
    """fl32(theta * theta): the single rounding of theta^2 used by the test."""
    return np.float32(float(theta) * float(theta))


def open_f32(gmin, gmax, c, h, theta: float) -> bool:
    """O4 for one (group box, cell cube) pair; True = open."""
    lib = _load()
    return bool(lib.ora_open_f32(np.asarray(gmin, np.float32), np.asarray(gmax, np.float32),
                                 np.asarray(c, np.float32), np.float32(h), theta2_f32(theta)))


def cell_field(com, M, S6, x, eps: float, G: float = 1.0):
    """O6 field of one cell (monopole + quadrupole) at point x: (acc[3], phi)."""
    lib = _load()
    a = np.zeros(3)
    p = np.zeros(1)
    lib.ora_cell_field(np.asarray(com, np.float64), float(M), np.asarray(S6, np.float64),
                       np.asarray(x, np.float64), float(eps) ** 2, float(G), a, p)
    return a, float(p[0])


class Tree:
    """O2/O3 tree of one system; keeps its own copies of pos and mass."""

    def __init__(self, pos, mass, n_leaf: int = 16, n_group: int | None = None,
                 max_depth: int = MAX_DEPTH):
        lib = _load()
        self.pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        self.mass = np.ascontiguousarray(mass, dtype=np.float64)
        self.n = self.mass.shape[0]
        self.n_leaf = int(n_leaf)
        self.n_group = int(n_group if n_group is not None else n_leaf)
        self._h = lib.ora_tree_build(self.pos.reshape(-1), self.mass, self.n, self.n_leaf,
                                     self.n_group, int(max_depth))
        if not self._h:
            raise ValueError("oracle tree build failed (bad arguments or out of memory)")
        info = np.zeros(6, np.int64)
        lib.ora_tree_info(self._h, info)
        self.n_cells, self.n_leaves, self.n_groups = int(info[1]), int(info[2]), int(info[3])
        self.max_depth, self.depth_reached = int(info[4]), int(info[5])
        fr = np.zeros(4)
        lib.ora_tree_frame(self._h, fr)
        self.lo, self.side = fr[:3].copy(), float(fr[3])
        nc = self.n_cells
        self.key = np.zeros(nc, np.uint64)
        self.depth = np.zeros(nc, np.int32)
        self.parent = np.zeros(nc, np.int64)
        self.leaf = np.zeros(nc, np.int32)
        self.first = np.zeros(nc, np.int64)
        self.count = np.zeros(nc, np.int64)
        self.child = np.zeros((nc, 8), np.int64)
        self.bmin = np.zeros((nc, 3))
        self.bmax = np.zeros((nc, 3))
        self.cube = np.zeros((nc, 4))
        self.M = np.zeros(nc)
        self.com = np.zeros((nc, 3))
        self.S = np.zeros((nc, 6))
        lib.ora_tree_cells(self._h, *[_ptr(a) for a in (
            self.key, self.depth, self.parent, self.leaf, self.first, self.count, self.child,
            self.bmin, self.bmax, self.cube, self.M, self.com, self.S)])
        self.members = np.zeros(self.n, np.int64)
        lib.ora_tree_members(self._h, self.members)
        self.groups = np.zeros(self.n_groups, np.int64)
        lib.ora_tree_groups(self._h, self.groups)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.ora_tree_free(h)
            self._h = None

    def cell_members(self, c: int) -> np.ndarray:
        f, k = int(self.first[c]), int(self.count[c])
        return self.members[f:f + k]

    def lists(self, g: int, theta: float):
        """O5: (cell-list cell indices, leaf-list cell indices) of group g."""
        lib = _load()
        cap = 1024
        while True:
            cells = np.zeros(cap, np.int64)
            leaves = np.zeros(cap, np.int64)
            nc = np.zeros(1, np.int64)
            nl = np.zeros(1, np.int64)
            tot = lib.ora_walk(self._h, int(g), float(theta), cells, cap, nc, leaves, cap, nl)
            if tot < 0:
                raise ValueError("oracle walk failed")
            if nc[0] <= cap and nl[0] <= cap:
                return cells[: nc[0]].copy(), leaves[: nl[0]].copy()
            cap = int(max(nc[0], nl[0]))

    def list_keys(self, g: int, theta: float):
        """O5 lists of group g as sorted multisets of layout-independent cell keys."""
        cells, leaves = self.lists(g, theta)
        return np.sort(self.key[cells]), np.sort(self.key[leaves])

    def forces(self, eps: float, theta: float, G: float = 1.0, groups=None,
               nthreads: int | None = None, counts: bool = True):
        """O6: acc [n,3], pot [n] (input order), n_pp [n], n_pc [n], fp32/fp64 flips.

        With ``groups`` given only those groups' particles are filled (others 0)."""
        lib = _load()
        acc = np.zeros((self.n, 3))
        pot = np.zeros(self.n)
        npp = np.zeros(self.n, np.int64) if counts else None
        npc = np.zeros(self.n, np.int64) if counts else None
        if groups is None:
            gp, ng, garr = None, self.n_groups, None
        else:
            garr = np.ascontiguousarray(groups, dtype=np.int64)
            gp, ng = garr.ctypes.data_as(C.c_void_p), garr.shape[0]
        flips = lib.ora_forces(self._h, float(eps), float(theta), float(G), gp, ng,
                               acc.reshape(-1), pot, _ptr(npp), _ptr(npc),
                               int(nthreads or default_threads()))
        if flips < 0:
            raise RuntimeError("oracle forces failed")
        return acc, pot, npp, npc, int(flips)

    # ---- O8: learned opening criterion
    def mlp_features(self, g: int, c: int) -> np.ndarray:
        f = np.zeros(12)
        _load().ora_mlp_features(self._h, int(g), int(c), f)
        return f

    def mlp_samples(self, groups, theta_walk: float, eps: float, aref, nthreads: int | None = None):
        """Features [S,12], labels [S] (relative error of accepting), pairs [S,2] (group, cell)."""
        lib = _load()
        garr = np.ascontiguousarray(groups, dtype=np.int64)
        aref = np.ascontiguousarray(aref, dtype=np.float64).reshape(-1)
        nt = int(nthreads or default_threads())
        tot = lib.ora_mlp_samples(self._h, garr, len(garr), float(theta_walk), float(eps), aref,
                                  None, None, None, 0, nt)
        feat = np.zeros((tot, 12))
        lab = np.zeros(tot)
        pair = np.zeros((tot, 2), np.int64)
        lib.ora_mlp_samples(self._h, garr, len(garr), float(theta_walk), float(eps), aref,
                            _ptr(feat), _ptr(lab), _ptr(pair), tot, nt)
        return feat, lab, pair

    def forces_mlp(self, eps: float, net: dict, tau: float, theta_lo: float, theta_hi: float, theta_fb: float,
                   G: float = 1.0, groups=None, nthreads: int | None = None, bf16: bool = False):
        """O6 with the learned criterion: acc, pot, n_pp, n_pc, number of network evaluations.
        bf16: evaluate the network with BF16 operands (mlp_forward_bf16)."""
        lib = _load()
        acc = np.zeros((self.n, 3))
        pot = np.zeros(self.n)
        npp = np.zeros(self.n, np.int64)
        npc = np.zeros(self.n, np.int64)
        if groups is None:
            gp, ng, garr = None, self.n_groups, None
        else:
            garr = np.ascontiguousarray(groups, dtype=np.int64)
            gp, ng = garr.ctypes.data_as(C.c_void_p), garr.shape[0]
        w = np.ascontiguousarray(net["w"], dtype=np.float64)
        args = [np.ascontiguousarray(net[k], dtype=np.float64) for k in ("mu", "sigma", "fmin", "fmax")]
        nm = lib.ora_forces_mlp(self._h, float(eps), float(G), w, *args, float(tau), float(theta_lo),
                                float(theta_hi), float(theta_fb), int(bf16), gp, ng, acc.reshape(-1), pot, _ptr(npp),
                                _ptr(npc), int(nthreads or default_threads()))
        if nm < 0:
            raise RuntimeError("oracle MLP forces failed")
        return acc, pot, npp, npc, int(nm)

    def mlp_decide(self, g: int, c: int, net: dict, tau: float, theta_lo: float, theta_hi: float,
                   theta_fb: float, bf16: bool = False):
        """One decision of the learned criterion for group g and cell c: (open, branch, y).

        branch: 0 the theta_hi test opens, 1 the theta_lo test accepts, 2 a
        point cell (h = 0) is accepted, 3 a standardised input is out of the
        training range and the theta_fb test decides, 4 the network decides
        (y = its prediction, accept iff y < tau; FP64, or with BF16 operands when bf16)."""
        w = np.ascontiguousarray(net["w"], dtype=np.float64)
        args = [np.ascontiguousarray(net[k], dtype=np.float64) for k in ("mu", "sigma", "fmin", "fmax")]
        br = C.c_int(0)
        y = C.c_double(0.0)
        op = _load().ora_mlp_decide(self._h, int(g), int(c), w, *args, float(tau), float(theta_lo),
                                    float(theta_hi), float(theta_fb), int(bf16), C.byref(br), C.byref(y))
        if op < 0:
            raise ValueError("group or cell index out of range")
        return bool(op), int(br.value), float(y.value)

    def mlp_decide_many(self, groups, cells, net: dict, tau: float, theta_lo: float, theta_hi: float,
                        theta_fb: float, features: bool = False, bf16: bool = False):
        """mlp_decide for pairs (groups[k], cells[k]): open [n] bool, branch [n], y [n] and, with
        ``features``, each pair's 12 inputs [n,12] (branches 3 and 4; zeros elsewhere)."""
        g = np.ascontiguousarray(groups, dtype=np.int64)
        c = np.ascontiguousarray(cells, dtype=np.int64)
        n = len(g)
        if len(c) != n:
            raise ValueError("groups and cells differ in length")
        w = np.ascontiguousarray(net["w"], dtype=np.float64)
        args = [np.ascontiguousarray(net[k], dtype=np.float64) for k in ("mu", "sigma", "fmin", "fmax")]
        op = np.zeros(n, np.int32)
        br = np.zeros(n, np.int32)
        y = np.zeros(n)
        f = np.zeros((n, 12)) if features else None
        rc = _load().ora_mlp_decide_many(self._h, n, g, c, w, *args, float(tau), float(theta_lo),
                                         float(theta_hi), float(theta_fb), int(bf16), op, br, y, _ptr(f))
        if rc < 0:
            raise ValueError("group or cell index out of range")
        return (op.astype(bool), br, y, f) if features else (op.astype(bool), br, y)

    def forces_on_lists(self, g: int, cells, leaves, eps: float, G: float = 1.0):
        """O6 for group g's particles (member order) from given cell and leaf lists (cell indices)."""
        n = int(self.count[self.groups[g]])
        acc = np.zeros((n, 3))
        pot = np.zeros(n)
        c = np.ascontiguousarray(cells, dtype=np.int64)
        lv = np.ascontiguousarray(leaves, dtype=np.int64)
        _load().ora_forces_on_lists(self._h, int(g), c, len(c), lv, len(lv), float(eps), float(G), acc.reshape(-1), pot)
        return acc, pot

    def group_of_particle(self) -> np.ndarray:
        """Group index of every particle (input order)."""
        out = np.full(self.n, -1, np.int64)
        for g, c in enumerate(self.groups):
            out[self.cell_members(int(c))] = g
        return out


def mlp_forward_c(w, x) -> float:
    """O8 FP64 forward pass (C) of the packed 12-64-64-1 network on one input."""
    return float(_load().ora_mlp_forward(np.ascontiguousarray(w, np.float64), np.ascontiguousarray(x, np.float64)))


def mlp_forward_bf16_c(w, x) -> float:
    """O8 forward pass with BF16 operands (inputs and first hidden layer rounded
    to BF16 by way of FP32; w must hold BF16 values where they multiply)."""
    return float(_load().ora_mlp_forward_bf16(np.ascontiguousarray(w, np.float64),
                                              np.ascontiguousarray(x, np.float64)))


def rel_err(a, a_ref):
    """Per-particle |a - a_ref| / |a_ref| (the paper's Delta a / a, Sec. 3.1)."""
    return np.linalg.norm(a - a_ref, axis=1) / np.linalg.norm(a_ref, axis=1)


def rel_rms(a, a_ref):
    """Global ||a - a_ref||_2 / ||a_ref||_2 over all listed particles."""
    return float(np.linalg.norm(a - a_ref) / np.linalg.norm(a_ref))
