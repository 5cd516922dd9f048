"""ctypes wrapper and build step for the plain FP64 C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and
the benchmark's CPU-baseline leg, never by the product package.  It shares
no code with the CUDA path.

Each wrapper returns numpy arrays; the C functions document which passage
of the paper (arXiv 2008.05712) they follow.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NONE32 = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = C.CDLL(_LIB)
            _declare(_lib)
    return _lib


P = C.c_void_p
I64 = C.c_int64


def _declare(L):
    L.orc_morton_keys.argtypes = [I64, P, P, P, P, P]
    L.orc_build_tree.argtypes = [I64, P, C.c_int, P, P, I64, P, P, P, P, P, P, P,
                                 P, P, I64, P, P, P, P, P]
    L.orc_walk.argtypes = [I64, P, P, P, P, P, P, P, P, P, I64, I64, I64, P, I64, P]
    L.orc_gravity.argtypes = [P, I64, P, I64, P, C.c_double, P]
    L.orc_gravity.restype = None
    L.orc_gravity_batch.argtypes = [P, I64, P, P, P, P, C.c_double, P]
    L.orc_gravity_batch.restype = None
    L.orc_md_cells.argtypes = [I64, P, I64, P, P]
    L.orc_md_tasks.argtypes = [I64, P, P, P, P]
    L.orc_md_tasks_2d.argtypes = [I64, P, P, P, P]
    L.orc_lj.argtypes = [P, I64, P, I64, P, C.c_int, P, I64, C.c_double, C.c_double,
                         I64, P, P]
    L.orc_residency.argtypes = [I64, I64, P, P, P, C.c_uint32, I64, P, P, P, P, P, P, P]
    L.orc_pack_perm.argtypes = [I64, P, P]
    L.orc_pack_perm.restype = None
    L.orc_pack_perm_batch.argtypes = [I64, P, P, P]
    L.orc_pack_perm_batch.restype = None
    L.orc_reduce.argtypes = [I64, P, P, P]
    L.orc_reduce.restype = None
    L.orc_kick_drift.argtypes = [I64, P, P, P, C.c_double]
    L.orc_kick_drift.restype = None
    L.orc_ewald.argtypes = [P, I64, P, I64, P, C.c_double, C.c_double, C.c_int, C.c_int, P]
    L.orc_ewald.restype = None


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def morton_keys(xyzm):
    x = _c(xyzm, np.float32)
    n = x.shape[0]
    keys = np.empty(n, np.uint64)
    q3 = np.empty((n, 3), np.uint32)
    lo = np.empty(3, np.float64)
    L = np.empty(1, np.float64)
    rc = lib().orc_morton_keys(n, _p(x), _p(keys), _p(q3), _p(lo), _p(L))
    assert rc == 0, rc
    return keys, q3, lo, float(L[0])


class Tree:
    """Octree built by the oracle (all arrays numpy)."""

    def __init__(self, xyzm, bucket_max=32):
        x = _c(xyzm, np.float32)
        n = x.shape[0]
        self.n = n
        cap = 2 * n + 64
        self.sorted_ids = np.empty(n, np.uint32)
        self.sorted_keys = np.empty(n, np.uint64)
        lvl = np.empty(cap, np.uint8)
        cell = np.empty((cap, 3), np.uint32)
        first = np.empty(cap, np.uint32)
        count = np.empty(cap, np.uint32)
        leaf = np.empty(cap, np.uint8)
        size = np.empty(cap, np.uint32)
        mono = np.empty((cap, 4), np.float64)
        child = np.empty((cap, 8), np.uint32)
        bf = np.empty(cap, np.uint32)
        bc = np.empty(cap, np.uint32)
        bn = np.empty(cap, np.uint32)
        bbox = np.empty((cap, 6), np.int32)
        nn = np.zeros(1, np.int64)
        nb = np.zeros(1, np.int64)
        rc = lib().orc_build_tree(n, _p(x), bucket_max, _p(self.sorted_ids),
                                  _p(self.sorted_keys), cap, _p(nn), _p(lvl), _p(cell),
                                  _p(first), _p(count), _p(leaf), _p(size), _p(mono),
                                  _p(child), cap, _p(nb), _p(bf), _p(bc), _p(bn),
                                  _p(bbox))
        assert rc == 0, rc
        k, b = int(nn[0]), int(nb[0])
        self.n_nodes, self.n_buckets = k, b
        self.level, self.cell, self.first = lvl[:k].copy(), cell[:k].copy(), first[:k].copy()
        self.count, self.leaf, self.size = count[:k].copy(), leaf[:k].copy(), size[:k].copy()
        self.mono, self.child = mono[:k].copy(), child[:k].copy()
        self.bucket_first, self.bucket_count = bf[:b].copy(), bc[:b].copy()
        self.bucket_node, self.bucket_box = bn[:b].copy(), bbox[:b].copy()

    def walk(self, bucket: int, theta_num: int, theta_den: int):
        cap = 4096
        while True:
            out = np.empty(cap, np.uint32)
            ln = np.zeros(1, np.int64)
            rc = lib().orc_walk(self.n, _p(self.level), _p(self.cell), _p(self.first),
                                _p(self.count), _p(self.leaf), _p(self.child),
                                _p(self.sorted_ids), _p(self.bucket_first),
                                _p(self.bucket_box), bucket, theta_num, theta_den,
                                _p(out), cap, _p(ln))
            if rc == 0:
                return out[:int(ln[0])].copy()
            assert rc == -1, rc
            cap = int(ln[0]) + 1

    def lists(self, theta_num: int, theta_den: int, buckets=None):
        """CSR interaction lists for the given buckets (all by default)."""
        if buckets is None:
            buckets = range(self.n_buckets)
        parts = [self.walk(int(b), theta_num, theta_den) for b in buckets]
        off = np.zeros(len(parts) + 1, np.uint64)
        off[1:] = np.cumsum([len(p) for p in parts])
        ids = np.concatenate(parts) if parts else np.empty(0, np.uint32)
        return off, ids.astype(np.uint32)

    def bucket_targets(self, buckets=None):
        if buckets is None:
            buckets = range(self.n_buckets)
        parts = [self.sorted_ids[self.bucket_first[b]:self.bucket_first[b] + self.bucket_count[b]]
                 for b in buckets]
        off = np.zeros(len(parts) + 1, np.uint64)
        off[1:] = np.cumsum([len(p) for p in parts])
        ids = np.concatenate(parts) if parts else np.empty(0, np.uint32)
        return off, ids.astype(np.uint32)

    def node_table(self):
        """float32 xyzm rows for node ids n + k: (com x, y, z, mass) rounded
        from the FP64 monopole."""
        t = np.empty((self.n_nodes, 4), np.float32)
        t[:, 0:3] = self.mono[:, 1:4]
        t[:, 3] = self.mono[:, 0]
        return t


def gravity(table, tgt, src, eps2):
    t = _c(table, np.float32)
    tg = _c(tgt, np.uint32)
    sr = _c(src, np.uint32)
    out = np.empty((tg.shape[0], 4), np.float64)
    lib().orc_gravity(_p(t), tg.shape[0], _p(tg), sr.shape[0], _p(sr), float(eps2), _p(out))
    return out


def gravity_batch(table, tgt_off, tgt, src_off, src, eps2):
    t = _c(table, np.float32)
    to, tg = _c(tgt_off, np.uint64), _c(tgt, np.uint32)
    so, sr = _c(src_off, np.uint64), _c(src, np.uint32)
    out = np.empty((tg.shape[0], 4), np.float64)
    lib().orc_gravity_batch(_p(t), to.shape[0] - 1, _p(to), _p(tg), _p(so), _p(sr),
                            float(eps2), _p(out))
    return out


def md_cells(cell_of_atom, ncell_total):
    c = _c(cell_of_atom, np.uint32)
    start = np.empty(ncell_total + 1, np.uint32)
    atoms = np.empty(c.shape[0], np.uint32)
    rc = lib().orc_md_cells(c.shape[0], _p(c), ncell_total, _p(start), _p(atoms))
    assert rc == 0, rc
    return start, atoms


def md_tasks(m):
    nt = 14 * m ** 3
    a = np.empty(nt, np.uint32)
    b = np.empty(nt, np.uint32)
    d = np.empty((nt, 3), np.int8)
    s = np.empty(nt, np.uint8)
    k = lib().orc_md_tasks(m, _p(a), _p(b), _p(d), _p(s))
    assert k == nt, k
    return a, b, d, s


def md_tasks_2d(m):
    nt = 5 * m ** 2
    a = np.empty(nt, np.uint32)
    b = np.empty(nt, np.uint32)
    d = np.empty((nt, 3), np.int8)
    s = np.empty(nt, np.uint8)
    k = lib().orc_md_tasks_2d(m, _p(a), _p(b), _p(d), _p(s))
    assert k == nt, k
    return a, b, d, s


def lj(table, a_ids, b_ids, is_self, d3, E, eps=1.0, sigma=1.0, rc2_grid=None):
    t = _c(table, np.float32)
    a = _c(a_ids, np.uint32)
    b = _c(b_ids, np.uint32) if b_ids is not None else np.empty(0, np.uint32)
    d = _c(d3, np.int8)
    outA = np.empty((a.shape[0], 4), np.float64)
    outB = np.empty((max(b.shape[0], 1), 4), np.float64)
    rc = lib().orc_lj(_p(t), a.shape[0], _p(a), b.shape[0], _p(b), int(bool(is_self)),
                      _p(d), int(E), float(eps), float(sigma), int(rc2_grid), _p(outA),
                      _p(outB))
    assert rc == 0, rc
    return outA, outB[:b.shape[0]]


class Residency:
    """Chare-table state driven by the oracle's deterministic policy."""

    def __init__(self, id_cap: int, cap: int):
        self.id_cap, self.cap = id_cap, cap
        self.slot_of_id = np.full(id_cap, NONE32, np.uint32)
        self.id_of_slot = np.full(cap, NONE32, np.uint32)
        self.last_use = np.zeros(cap, np.uint32)

    def flush(self, entry_ids, epoch: int):
        e = _c(entry_ids, np.uint32)
        n = e.shape[0]
        slots = np.empty(n, np.uint32)
        uniq = np.empty(max(n, 1), np.uint32)
        reuse = np.empty(max(n, 1), np.uint32)
        miss = np.empty(max(n, 1), np.uint32)
        evicted = np.empty(max(self.cap, 1), np.uint32)
        stats = np.zeros(4, np.int64)
        rc = lib().orc_residency(self.id_cap, self.cap, _p(self.slot_of_id),
                                 _p(self.id_of_slot), _p(self.last_use), epoch, n, _p(e),
                                 _p(slots), _p(uniq), _p(reuse), _p(miss), _p(evicted),
                                 _p(stats))
        if rc != 0:
            return rc, None
        h, m, ev, u = (int(v) for v in stats)
        return 0, dict(slots=slots, uniq=uniq[:u].copy(), reuse=reuse[:u].copy(),
                       miss=miss[:m].copy(), evicted=evicted[:ev].copy(), hits=h,
                       misses=m, evictions=ev, unique=u)


def pack_perm(slots):
    s = _c(slots, np.uint32)
    perm = np.empty(s.shape[0], np.uint32)
    lib().orc_pack_perm(s.shape[0], _p(s), _p(perm))
    return perm


def pack_perm_batch(off, slots):
    o = _c(off, np.uint64)
    s = _c(slots, np.uint32)
    perm = np.empty(s.shape[0], np.uint32)
    lib().orc_pack_perm_batch(o.shape[0] - 1, _p(o), _p(s), _p(perm))
    return perm


def reduce(ids, contrib, id_cap):
    i = _c(ids, np.uint32)
    c = _c(contrib, np.float64)
    tot = np.zeros((id_cap, 4), np.float64)
    lib().orc_reduce(i.shape[0], _p(i), _p(c), _p(tot))
    return tot


def kick_drift(acc, xyzm, vel, dt):
    """One leapfrog step (kick then drift); returns new (xyzm, vel)."""
    a = _c(acc, np.float64)
    x = np.array(xyzm, dtype=np.float32, copy=True, order="C")
    v = np.array(vel, dtype=np.float32, copy=True, order="C")
    lib().orc_kick_drift(x.shape[0], _p(a), _p(x), _p(v), float(dt))
    return x, v


def ewald(table, tgt, src, L, alpha=None, nrep=2, hcut2=10):
    """Ewald corrections (periodic minus plain point-mass term) of the
    targets from the sources, (nt, 4) FP64 (ax, ay, az, phi)."""
    t = _c(table, np.float32)
    a = _c(tgt, np.uint32)
    b = _c(src, np.uint32)
    out = np.zeros((a.shape[0], 4), np.float64)
    alpha = 2.0 / L if alpha is None else alpha
    lib().orc_ewald(_p(t), a.shape[0], _p(a), b.shape[0], _p(b), float(L), float(alpha),
                    int(nrep), int(hcut2), _p(out))
    return out
