"""Thin ctypes binding of liboctgrav.so (the C ABI in include/octgrav.h).

Argument marshalling only: every step of the force calculation runs inside the
library (FP64 octree build on the host or on the GPU, sm_103a walk + evaluation
kernel). There is no
Python or CPU fallback: if the library cannot be built or loaded, the calls
raise.

Device buffers and streams may come from PyTorch: ``Tree.forces_device``
accepts a CUDA tensor of shape [n, 4] (float32) as its output and the handle of
a torch stream (default: the current stream).
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import build as _build

OK = 0
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_STACK, ERR_LIST, ERR_TIMEOUT, ERR_NONFINITE, ERR_STATE, ERR_INDEX = \
    -1, -2, -3, -4, -5, -6, -7, -8, -9
MAX_DEPTH = 21
MAX_ITEM = 64
NOALLOC_MAX_ITEMS = 262144

_lock = threading.Lock()
_lib = None

_f64 = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_vp = C.c_void_p

# name -> (restype, argtypes)
_SIGS = {
    "octgrav_version": (C.c_int, []),
    "octgrav_last_error": (C.c_char_p, []),
    "octgrav_build_tree": (C.c_int, [_f64, _f64, C.c_int64, C.c_int, C.c_int, C.POINTER(_vp)]),
    "octgrav_build_batch": (C.c_int, [C.c_int, _i64, _f64, _f64, C.c_int, C.c_int, C.POINTER(_vp)]),
    "octgrav_tree_upload": (C.c_int, [_vp, _vp]),
    "octgrav_forces_device": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, _vp, _vp]),
    "octgrav_set_system_params": (C.c_int, [_vp, _vp, _vp]),
    "octgrav_forces_tree": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, _vp, _vp, _vp]),
    "octgrav_forces": (C.c_int, [_f64, _f64, C.c_int64, C.c_double, C.c_double, C.c_int, _vp, _vp]),
    "octgrav_forces_ex": (C.c_int, [_f64, _f64, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int,
                                    C.c_int, _vp, _vp, _vp]),
    "octgrav_build_tree_gpu": (C.c_int, [_vp, _vp, C.c_int64, C.c_int, C.c_int, _vp, C.POINTER(_vp)]),
    "octgrav_build_batch_gpu": (C.c_int, [C.c_int, _i64, _vp, _vp, C.c_int, C.c_int, _vp, C.POINTER(_vp)]),
    "octgrav_forces_tree_device64": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, _vp, _vp, _vp]),
    "octgrav_forces_gpu": (C.c_int, [_vp, _vp, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                     _vp, _vp, _vp]),
    "octgrav_sim_create": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int,
                                     C.c_int, _vp, C.POINTER(_vp)]),
    "octgrav_sim_step": (C.c_int, [_vp, C.c_double, C.c_int, _vp]),
    "octgrav_sim_energy": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double), _vp]),
    "octgrav_sim_state": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "octgrav_sim_free": (None, [_vp]),
    "octgrav_sim_set_rebuild": (C.c_int, [_vp, C.c_int]),
    "octgrav_refit_tree_gpu": (C.c_int, [_vp, _vp, _vp, _vp]),
    "octgrav_direct": (C.c_int, [_vp, _vp, C.c_int64, _vp, C.c_int64, C.c_double, C.c_double, _vp, _vp, _vp]),
    "octgrav_forces_batched": (C.c_int, [C.c_int, _i64, _vp, _vp, _f64, _f64, _vp, _vp, _vp]),
    "octgrav_forces_batched_ex": (C.c_int, [C.c_int, _i64, _vp, _vp, _f64, _f64, C.c_double, C.c_int, C.c_int,
                                            _vp, _vp, _vp]),
    "octgrav_status": (C.c_int, [_vp, _vp]),
    "octgrav_tree_stats": (C.c_int, [_vp, _i64, C.c_int]),
    "octgrav_tree_perm": (C.c_int, [_vp, _i64]),
    "octgrav_tree_cell_keys": (C.c_int, [_vp, _vp]),
    "octgrav_tree_cell_props": (C.c_int, [_vp] + [_vp] * 7),
    "octgrav_item_info": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "octgrav_interaction_counts": (C.c_int, [_vp, _i64, _vp]),
    "octgrav_debug_lists": (C.c_int, [_vp, C.c_double, C.c_int, _vp, _vp, _vp, _vp, _vp]),
    "octgrav_debug_walk": (C.c_int, [_vp, C.c_double, C.c_int64, _vp, C.c_int, _vp, _vp, _vp, _vp, C.c_int, _vp,
                                     _vp, _vp, _vp]),
    "octgrav_set_launch": (C.c_int, [_vp, C.c_int, C.c_int]),
    "octgrav_balance": (C.c_int, [_vp, C.c_int, _vp]),
    "octgrav_set_staging": (C.c_int, [_vp, C.c_int]),
    "octgrav_set_fault": (C.c_int, [_vp, C.c_int, C.c_int64]),
    "octgrav_set_split": (C.c_int, [_vp, C.c_int]),
    "octgrav_oneshot_phases": (C.c_int, [_vp, C.c_int]),
    "octgrav_mlp_samples": (C.c_int, [_vp, _i64, C.c_int64, C.c_double, C.c_double, _vp, _vp, _vp, C.c_int64,
                                      C.POINTER(C.c_int64), _vp]),
    "octgrav_mlp_train": (C.c_int, [_vp, _vp, C.c_int64, C.c_int, C.c_int, C.c_double, C.c_uint64, _vp, _vp,
                                    _vp]),
    "octgrav_mlp_grad": (C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, _vp, _vp]),
    "octgrav_set_criterion": (C.c_int, [_vp, _vp, C.c_double, C.c_double, C.c_double, C.c_double]),
    "octgrav_graph_capture": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, _vp, _vp]),
    "octgrav_graph_launch": (C.c_int, [_vp, _vp]),
    "octgrav_autotune": (C.c_int, [C.c_int, _i64, _f64, _f64, C.c_int, C.c_double, C.c_double, _vp, C.c_int,
                                   _vp, _vp, _vp]),
    "octgrav_autotune_ex": (C.c_int, [C.c_int, _i64, _f64, _f64, C.c_int, C.c_double, C.c_double, _vp, C.c_int,
                                      _vp, C.c_int, _vp, _vp]),
    "octgrav_free_tree": (None, [_vp]),
    "octgrav_forces_noalloc": (C.c_int, [_vp, _vp, C.POINTER(C.c_size_t), C.c_double, C.c_double, C.c_double,
                                         _vp, _vp]),
}


class OctgravError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("octgrav error %d: %s" % (code, msg))
        self.code = code


def load(path: str | None = None):
    """Build (if stale) and load liboctgrav.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(path or _build.build())
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def exported_symbols():
    return sorted(_SIGS)


def _check(rc: int):
    if rc != OK:
        raise OctgravError(rc, load().octgrav_last_error().decode(errors="replace"))


def _p(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _pm(pos, mass):
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    if pos.shape[0] != 3 * mass.shape[0]:
        raise ValueError("pos must have shape [n, 3] matching mass [n]")
    return pos, mass


class Tree:
    """An octgrav_tree handle (host FP64 tree + library-owned device arrays)."""

    def __init__(self, handle, n: int):
        self._h = C.c_void_p(handle)
        self.n = n
        self.stats = self._stats()

    # ---- construction
    @classmethod
    def build(cls, pos, mass, n_leaf: int = 16, n_group: int | None = None) -> "Tree":
        lib = load()
        pos, mass = _pm(pos, mass)
        h = C.c_void_p()
        _check(lib.octgrav_build_tree(pos, mass, mass.shape[0], int(n_leaf),
                                      int(n_group if n_group is not None else n_leaf), C.byref(h)))
        return cls(h.value, mass.shape[0])

    @classmethod
    def build_batch(cls, systems, n_leaf: int = 16, n_group: int | None = None) -> "Tree":
        """systems: list of (pos [n_s,3], mass [n_s]) pairs."""
        lib = load()
        pos = np.ascontiguousarray(np.concatenate([np.asarray(p, np.float64).reshape(-1, 3) for p, _ in systems]))
        mass = np.ascontiguousarray(np.concatenate([np.asarray(m, np.float64) for _, m in systems]))
        off = np.zeros(len(systems) + 1, np.int64)
        off[1:] = np.cumsum([len(m) for _, m in systems])
        h = C.c_void_p()
        _check(lib.octgrav_build_batch(len(systems), off, pos.reshape(-1), mass, int(n_leaf),
                                       int(n_group if n_group is not None else n_leaf), C.byref(h)))
        t = cls(h.value, int(off[-1]))
        t.offsets = off
        return t

    @classmethod
    def build_gpu(cls, pos, mass, n_leaf: int = 16, n_group: int | None = None, offsets=None,
                  stream=None) -> "Tree":
        """The same tree as build / build_batch, built on the GPU. pos [n,3] and
        mass [n] are float64 CUDA tensors or host arrays (copied to the device);
        offsets (host, n_sys + 1) makes it a batch of concatenated systems."""
        import torch
        lib = load()

        def dev(a, shape):
            if isinstance(a, torch.Tensor):
                a = a.to(device="cuda", dtype=torch.float64).contiguous()
            else:
                a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
            return a.reshape(shape)
        m = dev(mass, (-1,))
        x = dev(pos, (-1, 3))
        n = m.shape[0]
        if x.shape[0] != n:
            raise ValueError("pos must have shape [n, 3] matching mass [n]")
        h = C.c_void_p()
        ng = int(n_group if n_group is not None else n_leaf)
        st = _stream_handle(stream)
        if offsets is None:
            _check(lib.octgrav_build_tree_gpu(C.c_void_p(x.data_ptr()), C.c_void_p(m.data_ptr()), n, int(n_leaf), ng,
                                              st, C.byref(h)))
            return cls(h.value, n)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        _check(lib.octgrav_build_batch_gpu(len(off) - 1, off, C.c_void_p(x.data_ptr()), C.c_void_p(m.data_ptr()),
                                           int(n_leaf), ng, st, C.byref(h)))
        t = cls(h.value, n)
        t.offsets = off
        return t

    def refit(self, pos, mass, stream=None):
        """Refit a GPU-built tree to new positions / masses of the same particles
        (CUDA float64 tensors or host arrays, input order)."""
        import torch
        x = pos if isinstance(pos, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(pos, dtype=np.float64))
        mm = mass if isinstance(mass, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(mass, dtype=np.float64))
        x = x.to(device="cuda", dtype=torch.float64).contiguous()
        mm = mm.to(device="cuda", dtype=torch.float64).contiguous()
        _check(load().octgrav_refit_tree_gpu(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(mm.data_ptr()),
                                             _stream_handle(stream)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.octgrav_free_tree(h)
            self._h = None

    def free(self):
        self.__del__()

    # ---- introspection
    def _stats(self):
        out = np.zeros(8, np.int64)
        _check(load().octgrav_tree_stats(self._h, out, 8))
        keys = ("n", "n_cells", "n_leaves", "n_groups", "n_items", "depth", "n_sys", "max_group")
        return dict(zip(keys, (int(v) for v in out)))

    def perm(self) -> np.ndarray:
        out = np.zeros(self.n, np.int64)
        _check(load().octgrav_tree_perm(self._h, out))
        return out

    def cell_keys(self) -> np.ndarray:
        out = np.zeros(self.stats["n_cells"], np.uint64)
        _check(load().octgrav_tree_cell_keys(self._h, _p(out)))
        return out

    def cell_props(self) -> dict:
        nc = self.stats["n_cells"]
        d = dict(bmin=np.zeros((nc, 3)), bmax=np.zeros((nc, 3)), cube=np.zeros((nc, 4)), mass=np.zeros(nc),
                 com=np.zeros((nc, 3)), S=np.zeros((nc, 6)), count=np.zeros(nc, np.int64))
        _check(load().octgrav_tree_cell_props(self._h, *[_p(d[k]) for k in
                                                         ("bmin", "bmax", "cube", "mass", "com", "S", "count")]))
        return d

    def item_info(self) -> dict:
        ni = self.stats["n_items"]
        d = dict(group_key=np.zeros(ni, np.uint64), first=np.zeros(ni, np.int64), count=np.zeros(ni, np.int32),
                 sys=np.zeros(ni, np.int32))
        _check(load().octgrav_item_info(self._h, _p(d["group_key"]), _p(d["first"]), _p(d["count"]), _p(d["sys"])))
        return d

    # ---- configuration
    def set_launch(self, particles_per_lane: int = 2, ctas_per_sm: int = 0):
        _check(load().octgrav_set_launch(self._h, int(particles_per_lane), int(ctas_per_sm)))
        self.stats = self._stats()

    def balance(self, mode: int = 1, stream=None):
        """Work-item order of later launches: longest first by the last launch's
        costs (1), most particles first (2, every new tree's default) or tree order (0)."""
        _check(load().octgrav_balance(self._h, int(mode), _stream_handle(stream)))

    def set_staging(self, mode: int):
        """0 = cp.async.bulk per record, 1 = 16-byte cp.async (default), 2 = TMA gather4."""
        _check(load().octgrav_set_staging(self._h, int(mode)))

    def set_split(self, nparts: int = 1):
        """Walk every work item with nparts warps, each evaluating a share of the
        lists (small systems; 1 = off)."""
        _check(load().octgrav_set_split(self._h, int(nparts)))

    def set_fault(self, stack_cap: int = 0, drop_item: int = -1):
        """Failure injection for tests: a node stack of stack_cap entries (0 = all),
        and (staging 2) a work item whose first tile is never requested (-1 = none)."""
        _check(load().octgrav_set_fault(self._h, int(stack_cap), int(drop_item)))

    def set_system_params(self, eps=None, theta=None):
        if eps is None and theta is None:
            _check(load().octgrav_set_system_params(self._h, None, None))
            return
        e = np.ascontiguousarray(eps, dtype=np.float64)
        t = np.ascontiguousarray(theta, dtype=np.float64)
        self._sysp_keep = (e, t)
        _check(load().octgrav_set_system_params(self._h, _p(e), _p(t)))

    # ---- device work
    def upload(self, stream=None):
        _check(load().octgrav_tree_upload(self._h, _stream_handle(stream)))

    def forces_device(self, eps: float, theta: float, out, G: float = 1.0, stream=None):
        """Launch on the GPU; ``out`` is a CUDA float32 tensor [n, 4] (tree order) or a raw pointer."""
        ptr = out if isinstance(out, int) else out.data_ptr()
        _check(load().octgrav_forces_device(self._h, float(eps), float(theta), float(G), C.c_void_p(ptr),
                                            _stream_handle(stream)))

    def forces(self, eps: float, theta: float, G: float = 1.0, stream=None):
        """Host outputs in input order: (acc [n,3], pot [n]) as float64 arrays."""
        acc = np.zeros((self.n, 3))
        pot = np.zeros(self.n)
        _check(load().octgrav_forces_tree(self._h, float(eps), float(theta), float(G), _p(acc), _p(pot),
                                          _stream_handle(stream)))
        return acc, pot

    def forces_device64(self, eps: float, theta: float, acc, pot=None, G: float = 1.0, stream=None):
        """Input-order FP64 results on the device: acc a CUDA float64 tensor [n,3],
        pot [n] or None. Enqueued only; check status()."""
        _check(load().octgrav_forces_tree_device64(self._h, float(eps), float(theta), float(G),
                                                   C.c_void_p(acc.data_ptr()),
                                                   None if pot is None else C.c_void_p(pot.data_ptr()),
                                                   _stream_handle(stream)))

    def noalloc_arena_bytes(self) -> int:
        """Device bytes the caller must provide to forces_noalloc for this tree."""
        need = C.c_size_t(0)
        _check(load().octgrav_forces_noalloc(self._h, None, C.byref(need), 1.0, 0.5, 1.0, None, None))
        return int(need.value)

    def forces_noalloc(self, eps: float, theta: float, out, arena, G: float = 1.0, stream=None):
        """Allocation-free launch: ``arena`` is caller-owned device memory (a CUDA
        uint8 tensor of at least noalloc_arena_bytes() bytes, or (pointer, size));
        ``out`` as for forces_device. Waits for the stream."""
        if isinstance(arena, tuple):
            ptr, size = arena
        else:
            ptr, size = arena.data_ptr(), arena.numel() * arena.element_size()
        optr = out if isinstance(out, int) else out.data_ptr()
        sz = C.c_size_t(size)
        _check(load().octgrav_forces_noalloc(self._h, C.c_void_p(ptr), C.byref(sz), float(eps), float(theta),
                                             float(G), C.c_void_p(optr), _stream_handle(stream)))

    # ---- learned opening criterion
    def mlp_samples(self, groups, theta_walk: float, eps: float, stream=None):
        """(features [S,12] float32, labels [S] float32, pairs [S,2] (group, cell))."""
        lib = load()
        g = np.ascontiguousarray(groups, dtype=np.int64)
        n = C.c_int64(0)
        _check(lib.octgrav_mlp_samples(self._h, g, len(g), float(theta_walk), float(eps), None, None, None, 0,
                                       C.byref(n), _stream_handle(stream)))
        f = np.zeros((n.value, 12), np.float32)
        lab = np.zeros(n.value, np.float32)
        pr = np.zeros((n.value, 2), np.int64)
        _check(lib.octgrav_mlp_samples(self._h, g, len(g), float(theta_walk), float(eps), _p(f), _p(lab), _p(pr),
                                       n.value, C.byref(n), _stream_handle(stream)))
        return f, lab, pr

    def set_criterion(self, record=None, tau: float = -3.5, theta_lo: float = 0.5, theta_hi: float = 4.0,
                      theta_fb: float = 1.0):
        """Enable the learned criterion (record from mlp_train) or restore the plain test (None).
        Switching between the two cuts the work items again (n_items may change)."""
        if record is None:
            _check(load().octgrav_set_criterion(self._h, None, 0.0, 0.0, 0.0, 0.0))
        else:
            r = np.ascontiguousarray(record, dtype=np.float32)
            _check(load().octgrav_set_criterion(self._h, _p(r), float(tau), float(theta_lo), float(theta_hi),
                                                float(theta_fb)))
        self.stats = self._stats()

    def capture_graph(self, eps: float, theta: float, out, G: float = 1.0, stream=None):
        """Capture one forces_device call into a CUDA graph (needs a non-default stream)."""
        ptr = out if isinstance(out, int) else out.data_ptr()
        _check(load().octgrav_graph_capture(self._h, float(eps), float(theta), float(G), C.c_void_p(ptr),
                                            _stream_handle(stream)))

    def launch_graph(self, stream=None):
        _check(load().octgrav_graph_launch(self._h, _stream_handle(stream)))

    def status(self, stream=None) -> int:
        return int(load().octgrav_status(self._h, _stream_handle(stream)))

    def interaction_counts(self, stream=None) -> dict:
        out = np.zeros(3, np.int64)
        _check(load().octgrav_interaction_counts(self._h, out, _stream_handle(stream)))
        return dict(n_pp=int(out[0]), n_pc=int(out[1]), flops=int(out[2]))

    def debug_lists(self, theta: float, cap: int = 8192, stream=None):
        """Per work item: (sorted cell-list keys, sorted leaf-list keys)."""
        ni = self.stats["n_items"]
        ck = np.zeros((ni, cap), np.uint64)
        lk = np.zeros((ni, cap), np.uint64)
        nc = np.zeros(ni, np.int32)
        nl = np.zeros(ni, np.int32)
        _check(load().octgrav_debug_lists(self._h, float(theta), int(cap), _p(ck), _p(nc), _p(lk), _p(nl),
                                          _stream_handle(stream)))
        return [(np.sort(ck[k, :nc[k]]), np.sort(lk[k, :nl[k]])) for k in range(ni)]

    def debug_walk(self, theta: float, items=None, cap: int = 8192, net_cap: int = 0, stream=None):
        """Capture the lists of the given work items (all when None). Returns one
        dict per requested item: 'cells' and 'leaves' (sorted key arrays) and,
        with net_cap > 0, 'net_keys' / 'net_y' (network candidates in walk
        order; y = NaN where the inputs were out of range)."""
        lib = load()
        if items is None:
            ns, ip = self.stats["n_items"], None
        else:
            arr = np.ascontiguousarray(items, dtype=np.int64)
            ns, ip = len(arr), _p(arr)
        ck = np.zeros((ns, cap), np.uint64)
        lk = np.zeros((ns, cap), np.uint64)
        nc = np.zeros(ns, np.int32)
        nl = np.zeros(ns, np.int32)
        nk = np.zeros((ns, max(net_cap, 1)), np.uint64)
        ny = np.zeros((ns, max(net_cap, 1)), np.float32)
        nn = np.zeros(ns, np.int32)
        _check(lib.octgrav_debug_walk(self._h, float(theta), ns, ip, int(cap), _p(ck), _p(nc), _p(lk), _p(nl),
                                      int(net_cap), _p(nk) if net_cap else None, _p(ny) if net_cap else None,
                                      _p(nn) if net_cap else None, _stream_handle(stream)))
        out = []
        for r in range(ns):
            d = dict(cells=np.sort(ck[r, :nc[r]]), leaves=np.sort(lk[r, :nl[r]]))
            if net_cap:
                d["net_keys"] = nk[r, :nn[r]].copy()
                d["net_y"] = ny[r, :nn[r]].copy()
            out.append(d)
        return out


def _out_arrays(n, out):
    if out is None:
        return np.zeros((n, 3)), np.zeros(n)
    acc, pot = out
    if acc.dtype != np.float64 or not acc.flags.c_contiguous or acc.size != 3 * n:
        raise ValueError("acc must be a C-contiguous float64 array of n x 3")
    if pot is not None and (pot.dtype != np.float64 or not pot.flags.c_contiguous or pot.size != n):
        raise ValueError("pot must be a C-contiguous float64 array of n")
    return acc, pot


def forces(pos, mass, eps: float, theta: float, n_leaf: int = 16, n_group: int | None = None, G: float = 1.0,
           stream=None, out=None):
    """One-shot C-ABI call with host buffers and the tree built on the host:
    (acc [n,3], pot [n]) in input order. ``out`` = (acc, pot) host float64
    arrays to fill (e.g. views of pinned memory)."""
    lib = load()
    pos, mass = _pm(pos, mass)
    n = mass.shape[0]
    acc, pot = _out_arrays(n, out)
    _check(lib.octgrav_forces_ex(pos, mass, n, float(eps), float(theta), float(G), int(n_leaf),
                                 int(n_group if n_group is not None else n_leaf), _p(acc), _p(pot),
                                 _stream_handle(stream)))
    return acc, pot


ONESHOT_PHASES = ("bbox_check", "morton", "sort", "gather_records", "levels", "cell_props", "groups",
                  "records_items", "host_build", "device_upload", "device_walk_eval", "device_unpermute_copy_out",
                  "call")


def oneshot_phases() -> dict:
    """Where the calling thread's last forces() call spent its time (ms)."""
    ms = np.zeros(len(ONESHOT_PHASES))
    k = load().octgrav_oneshot_phases(_p(ms), len(ms))
    if k < 0:
        _check(k)
    return {name: float(ms[i]) for i, name in enumerate(ONESHOT_PHASES[:k])}


def forces_gpu(pos, mass, eps: float, theta: float, n_leaf: int = 16, n_group: int | None = None, G: float = 1.0,
               stream=None, out=None):
    """One-shot C-ABI call with host buffers and the tree built on the GPU:
    (acc [n,3], pot [n]) in input order. ``out`` = (acc, pot) host float64
    arrays to fill (e.g. views of pinned memory); pos / mass should be pinned
    too for link-speed copies."""
    lib = load()
    pos, mass = _pm(pos, mass)
    n = mass.shape[0]
    acc, pot = _out_arrays(n, out)
    _check(lib.octgrav_forces_gpu(_p(pos), _p(mass), n, float(eps), float(theta), float(G), int(n_leaf),
                                  int(n_group if n_group is not None else n_leaf), _p(acc), _p(pot),
                                  _stream_handle(stream)))
    return acc, pot


def forces_batched(systems, eps, theta, G: float = 1.0, n_leaf: int = 16, n_group: int = 256, out=None,
                   stream=None):
    """One-shot forces of many independent systems through octgrav_forces_batched_ex.

    ``systems`` is a list of (pos [n_s,3], mass [n_s]) or a tuple (offsets, pos, mass)
    of concatenated host arrays; ``eps`` and ``theta`` are scalars or one value
    per system. Returns (acc [n,3], pot [n]) in input order. ``out`` may give
    (acc, pot) host arrays (e.g. pinned torch tensors' numpy views) to fill."""
    if isinstance(systems, tuple):
        off, pos, mass = systems
        off = np.ascontiguousarray(off, np.int64)
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        mass = np.ascontiguousarray(mass, np.float64)
    else:
        off = np.zeros(len(systems) + 1, np.int64)
        off[1:] = np.cumsum([len(m) for _, m in systems])
        pos = np.ascontiguousarray(np.concatenate([p for p, _ in systems]), np.float64)
        mass = np.ascontiguousarray(np.concatenate([m for _, m in systems]), np.float64)
    ns = len(off) - 1
    e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, np.float64), (ns,)))
    t = np.ascontiguousarray(np.broadcast_to(np.asarray(theta, np.float64), (ns,)))
    n = int(off[-1])
    acc, pot = out if out is not None else (np.empty((n, 3)), np.empty(n))
    _check(load().octgrav_forces_batched_ex(ns, off, pos.ctypes.data_as(_vp), mass.ctypes.data_as(_vp), e, t,
                                            float(G), int(n_leaf), int(n_group), acc.ctypes.data_as(_vp),
                                            None if pot is None else pot.ctypes.data_as(_vp),
                                            _stream_handle(stream)))
    return acc, pot


def direct(pos, mass, eps: float, G: float = 1.0, targets=None, stream=None):
    """FP64 direct summation on the GPU at ``targets`` (all particles when
    None): (acc [nt,3], pot [nt]); the reference of the error measurements."""
    lib = load()
    pos, mass = _pm(pos, mass)
    n = mass.shape[0]
    if targets is None:
        t, nt = None, n
    else:
        t = np.ascontiguousarray(targets, dtype=np.int64)
        nt = t.shape[0]
    acc = np.zeros((nt, 3))
    pot = np.zeros(nt)
    _check(lib.octgrav_direct(_p(pos), _p(mass), n, _p(t), nt, float(eps), float(G), _p(acc), _p(pot),
                              _stream_handle(stream)))
    return acc, pot


def rel_err(a, a_ref):
    """Per-particle |a - a_ref| / |a_ref| (the paper's Delta a / a)."""
    return np.linalg.norm(np.asarray(a) - a_ref, axis=1) / np.linalg.norm(a_ref, axis=1)


class Sim:
    """Leapfrog (kick-drift-kick) integrator with the state on the GPU and the
    tree rebuilt on the GPU at every force evaluation."""

    def __init__(self, pos, vel, mass, eps: float, theta: float, G: float = 1.0, n_leaf: int = 16,
                 n_group: int | None = None, stream=None):
        lib = load()
        pos, mass = _pm(pos, mass)
        vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1)
        if vel.shape != pos.shape:
            raise ValueError("vel must have the shape of pos")
        self.n = mass.shape[0]
        h = C.c_void_p()
        _check(lib.octgrav_sim_create(_p(pos), _p(vel), _p(mass), self.n, float(eps), float(theta), float(G),
                                      int(n_leaf), int(n_group if n_group is not None else n_leaf),
                                      _stream_handle(stream), C.byref(h)))
        self._h = h

    def set_rebuild(self, every: int):
        """Full tree build every `every` force evaluations, refits in between."""
        _check(load().octgrav_sim_set_rebuild(self._h, int(every)))

    def step(self, dt: float, n_steps: int = 1, stream=None):
        _check(load().octgrav_sim_step(self._h, float(dt), int(n_steps), _stream_handle(stream)))

    def energy(self, stream=None):
        """(kinetic, potential) in FP64."""
        k, w = C.c_double(), C.c_double()
        _check(load().octgrav_sim_energy(self._h, C.byref(k), C.byref(w), _stream_handle(stream)))
        return k.value, w.value

    def state(self, stream=None):
        """(pos, vel, acc [n,3], pot [n]) on the host."""
        x, v, a = np.zeros((self.n, 3)), np.zeros((self.n, 3)), np.zeros((self.n, 3))
        p = np.zeros(self.n)
        _check(load().octgrav_sim_state(self._h, _p(x), _p(v), _p(a), _p(p), _stream_handle(stream)))
        return x, v, a, p

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.octgrav_sim_free(h)
            self._h = None


MLP_RECORD = 5105
MLP_NPARAM = 5057


def mlp_train(features, labels, steps: int = 3000, batch: int = 4096, lr: float = 2e-3, seed: int = 1,
              stream=None):
    """Train the criterion's network on the GPU; returns (record [5105] float32, last loss)."""
    f = np.ascontiguousarray(features, dtype=np.float32)
    lab = np.ascontiguousarray(labels, dtype=np.float32)
    rec = np.zeros(MLP_RECORD, np.float32)
    loss = np.zeros(1, np.float32)
    _check(load().octgrav_mlp_train(_p(f), _p(lab), len(lab), int(steps), int(batch), float(lr), int(seed),
                                    _p(rec), _p(loss), _stream_handle(stream)))
    return rec, float(loss[0])


CRITERION_FORMAT = "octgrav-criterion-1"


def save_criterion(path, record, tau: float, theta_lo: float, theta_hi: float, theta_fb: float, **meta):
    """Save a trained criterion -- the FP32 record of mlp_train (input scaling,
    training range, network) with the tau and theta band it is used with -- to
    an .npz file. ``meta`` holds free-form scalars or strings (training system,
    seed, ...). The network is rounded to BF16 only when the record is set on a
    tree, so the file keeps the trained FP32 values."""
    rec = np.ascontiguousarray(record, dtype=np.float32)
    if rec.shape != (MLP_RECORD,) or not np.all(np.isfinite(rec[:24])):
        raise ValueError("not a criterion record of %d floats" % MLP_RECORD)
    band = np.array([tau, theta_lo, theta_hi, theta_fb], np.float64)
    if not np.all(np.isfinite(band)):
        raise ValueError("tau and the theta band must be finite")
    np.savez(path, format=np.array(CRITERION_FORMAT), record=rec, band=band,
             meta_keys=np.array(list(meta.keys()), dtype=str),
             meta_values=np.array([str(v) for v in meta.values()], dtype=str))


def load_criterion(path) -> dict:
    """Load a criterion saved by save_criterion: dict(record, tau, theta_lo,
    theta_hi, theta_fb, meta); ``Tree.set_criterion(**{k: d[k] for k in ...})``
    applies it. Raises ValueError on a file of another format."""
    with np.load(path, allow_pickle=False) as z:
        if "format" not in z.files or str(z["format"]) != CRITERION_FORMAT:
            raise ValueError("%s is not an octgrav criterion file" % path)
        rec = z["record"].astype(np.float32)
        if rec.shape != (MLP_RECORD,):
            raise ValueError("criterion record has %d floats, expected %d" % (rec.size, MLP_RECORD))
        tau, lo, hi, fb = (float(v) for v in z["band"])
        meta = dict(zip((str(k) for k in z["meta_keys"]), (str(v) for v in z["meta_values"])))
    return dict(record=rec, tau=tau, theta_lo=lo, theta_hi=hi, theta_fb=fb, meta=meta)


def mlp_grad(params, x, t, stream=None):
    """GPU gradient of sum (y - t)^2 / (2n) at params over standardised inputs x [n,12]: (grad, loss)."""
    w = np.ascontiguousarray(params, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float32)
    tt = np.ascontiguousarray(t, dtype=np.float32)
    g = np.zeros(MLP_NPARAM, np.float32)
    loss = np.zeros(1, np.float32)
    _check(load().octgrav_mlp_grad(_p(w), _p(xx), _p(tt), len(tt), _p(g), _p(loss), _stream_handle(stream)))
    return g, float(loss[0])


def autotune(systems, n_leaf: int = 16, eps: float = 0.01, theta: float = 0.5, candidates=(16, 32, 64, 128),
             staging: bool = True, stream=None) -> dict:
    """Pick n_group, particles-per-lane, list split and (with ``staging``) the
    staging mode of the cell records by timing the kernel on these systems.

    systems: list of (pos [n_s,3], mass [n_s]) pairs (one pair for a single system)."""
    lib = load()
    pos = np.ascontiguousarray(np.concatenate([np.asarray(p, np.float64).reshape(-1, 3) for p, _ in systems]))
    mass = np.ascontiguousarray(np.concatenate([np.asarray(m, np.float64) for _, m in systems]))
    off = np.zeros(len(systems) + 1, np.int64)
    off[1:] = np.cumsum([len(m) for _, m in systems])
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    best = np.zeros(4, np.int32)
    best[3] = 1
    ms = np.zeros(1)
    if staging:
        _check(lib.octgrav_autotune_ex(len(systems), off, pos.reshape(-1), mass, int(n_leaf), float(eps),
                                       float(theta), _p(cand), len(cand), _p(best), 4, _p(ms),
                                       _stream_handle(stream)))
    else:
        _check(lib.octgrav_autotune(len(systems), off, pos.reshape(-1), mass, int(n_leaf), float(eps),
                                    float(theta), _p(cand), len(cand), _p(best), _p(ms), _stream_handle(stream)))
    return dict(n_group=int(best[0]), particles_per_lane=int(best[1]), split=int(best[2]), staging=int(best[3]),
                ms=float(ms[0]))


def version() -> int:
    return int(load().octgrav_version())
