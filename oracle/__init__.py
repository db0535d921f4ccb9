"""ctypes view of the SCO oracle (test infrastructure only).

The oracle is a plain CPU C restatement of the parallelized stochastic cutoff
method (Endo, Toga and Sasaki, arXiv:1503.03295) used to check the CUDA
library.  Only tests, the smoke check and the CPU-baseline leg of the
benchmark may import this package; the product never does.
"""
import ctypes as C
import math

import numpy as np

from . import build as _build

TAG_INIT, TAG_SWITCH, TAG_PROPOSE, TAG_DIRECT, TAG_PLAIN = 1, 2, 3, 4, 5
EXCH_ONLY = 0x80000000


class Params(C.Structure):
    _fields_ = [("Lx", C.c_int32), ("Ly", C.c_int32), ("J", C.c_double), ("D", C.c_double),
                ("T", C.c_double), ("seed", C.c_uint64), ("n_sw", C.c_int32),
                ("colour_variant", C.c_int32), ("replica", C.c_int32), ("pad", C.c_int32)]


class Obs(C.Structure):
    _fields_ = [("e_switched", C.c_double), ("e_exchange", C.c_double), ("e_full", C.c_double),
                ("mx", C.c_double), ("my", C.c_double), ("mz", C.c_double),
                ("m_abs", C.c_double), ("m_phi", C.c_double), ("n_edges", C.c_int64),
                ("max_degree", C.c_int32), ("n_colours", C.c_int32), ("kw_rounds", C.c_int32),
                ("max_degree_dipolar", C.c_int32), ("sweeps_done", C.c_int64),
                ("guard_hits", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GraphStats(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("n_cross", C.c_int64), ("p_ipc", C.c_double),
                ("delta_r_mean", C.c_double), ("delta_r_max", C.c_double),
                ("delta_r_weighted", C.c_double), ("n_cells", C.c_int32), ("palette", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_P = np.ctypeslib.ndpointer


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        vp = C.c_void_p
        L.sco_ref_philox.argtypes = [_P(np.uint64, flags="C"), _P(np.uint64, flags="C"),
                                     _P(np.uint64, flags="C")]
        L.sco_ref_marsaglia.argtypes = [C.c_uint64, C.c_uint64, _P(np.float64, flags="C")]
        L.sco_ref_marsaglia.restype = C.c_int
        L.sco_ref_table_size.argtypes = [C.c_int32, C.c_int32]
        L.sco_ref_table_size.restype = C.c_int64
        L.sco_ref_table.argtypes = [C.c_int32, C.c_int32] + [vp] * 6
        L.sco_ref_pair_V.argtypes = [C.c_double, _P(np.float64, flags="C"),
                                     _P(np.float64, flags="C"), C.c_int32, C.c_int32]
        L.sco_ref_pair_V.restype = C.c_double
        L.sco_ref_vmax.argtypes = [C.c_double, C.c_int64]
        L.sco_ref_vmax.restype = C.c_double
        for f in ("sco_ref_switch_prob", "sco_ref_pseudo"):
            getattr(L, f).argtypes = [C.c_double] * 3
            getattr(L, f).restype = C.c_double
        L.sco_ref_init.argtypes = [C.POINTER(Params), C.POINTER(vp)]
        L.sco_ref_destroy.argtypes = [vp]
        L.sco_ref_switch.argtypes = [vp]
        L.sco_ref_switch_epoch.argtypes = [vp, C.c_uint32]
        L.sco_ref_colour.argtypes = [vp, C.POINTER(C.c_int32)]
        L.sco_ref_sweep.argtypes = [vp, C.c_int32]
        L.sco_ref_run_series.argtypes = [vp, C.c_int64, vp, vp]
        L.sco_ref_observables.argtypes = [vp, C.POINTER(Obs), C.c_int32]
        for f in ("sco_ref_n_sites", "sco_ref_n_entries", "sco_ref_n_half_edges",
                  "sco_ref_sweeps_done"):
            getattr(L, f).argtypes = [vp]
            getattr(L, f).restype = C.c_int64
        L.sco_ref_get_spins.argtypes = [vp, vp]
        L.sco_ref_set_spins.argtypes = [vp, vp]
        L.sco_ref_get_graph.argtypes = [vp, vp, vp, vp]
        L.sco_ref_get_edges.argtypes = [vp, vp, vp, vp, vp]
        L.sco_ref_get_classes.argtypes = [vp, vp, vp]
        L.sco_ref_get_accepts.argtypes = [vp, vp]
        L.sco_ref_set_threads.argtypes = [C.c_int32]
        L.sco_ref_set_guard_scale.argtypes = [C.c_double]
        L.sco_ref_kw_colour_graph.argtypes = [C.c_int64, vp, vp, C.c_int32, vp,
                                              C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.sco_ref_direct_switch.argtypes = [vp, C.c_uint32, vp]
        L.sco_ref_plain_metropolis.argtypes = [C.POINTER(Params), vp, C.c_int64, vp, vp, vp]
        L.sco_ref_full_energy.argtypes = [C.POINTER(Params), vp]
        L.sco_ref_full_energy.restype = C.c_double
        L.sco_ref_set_temperature.argtypes = [vp, C.c_double]
        L.sco_ref_graph_stats.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32,
                                          C.POINTER(GraphStats), vp, vp, vp, vp]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _check(st, what):
    if st != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, st))


def make_params(Lx, Ly=None, T=1.0, D=1.0, J=0.0, seed=0, n_sw=1, colour_variant=0, replica=0):
    return Params(Lx, Lx if Ly is None else Ly, J, D, T, seed, n_sw, colour_variant, replica, 0)


def set_threads(n):
    lib().sco_ref_set_threads(int(n))


def set_guard_scale(s):
    lib().sco_ref_set_guard_scale(float(s))


# ---- stateless pieces ----------------------------------------------------------------
def philox(ctr, key):
    out = np.zeros(4, np.uint64)
    lib().sco_ref_philox(np.ascontiguousarray(ctr, np.uint64),
                         np.ascontiguousarray(key, np.uint64), out)
    return out


def marsaglia(w0, w1):
    S = np.zeros(3)
    ok = lib().sco_ref_marsaglia(int(w0), int(w1), S)
    return (S if ok else None)


def table(Lx, Ly=None):
    Ly = Lx if Ly is None else Ly
    K = lib().sco_ref_table_size(Lx, Ly)
    out = dict(dx=np.zeros(K, np.int32), dy=np.zeros(K, np.int32), r2=np.zeros(K, np.int64),
               c=np.zeros(K), A=np.zeros(K, np.uint64), W=np.zeros(K, np.uint64))
    _check(lib().sco_ref_table(Lx, Ly, *[_ptr(out[k]) for k in ("dx", "dy", "r2", "c", "A", "W")]),
           "table")
    return out


def pair_V(D, Si, Sj, dx, dy):
    return lib().sco_ref_pair_V(D, np.ascontiguousarray(Si, float), np.ascontiguousarray(Sj, float),
                                dx, dy)


def vmax(D, r2):
    return lib().sco_ref_vmax(D, int(r2))


def switch_prob(beta, V, Vmax):
    return lib().sco_ref_switch_prob(beta, V, Vmax)


def pseudo(beta, V, Vmax):
    return lib().sco_ref_pseudo(beta, V, Vmax)


def kw_colour_graph(row_ptr, col, variant=0):
    """KW colouring of a symmetric CSR graph; returns (colour, rounds, max_degree)."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.uint32)
    N = len(row_ptr) - 1
    colour = np.zeros(max(N, 1), np.int32)
    rounds, delta = C.c_int32(0), C.c_int32(0)
    _check(lib().sco_ref_kw_colour_graph(N, _ptr(row_ptr), _ptr(col), variant, _ptr(colour),
                                         C.byref(rounds), C.byref(delta)), "kw")
    return colour[:N], rounds.value, delta.value


def full_energy(params, xyz):
    xyz = np.ascontiguousarray(xyz, np.float64)
    return lib().sco_ref_full_energy(C.byref(params), _ptr(xyz))


def plain_metropolis(params, xyz0, n_mcs):
    xyz0 = np.ascontiguousarray(xyz0, np.float64)
    e = np.zeros(n_mcs)
    m = np.zeros(n_mcs)
    out = np.zeros_like(xyz0)
    _check(lib().sco_ref_plain_metropolis(C.byref(params), _ptr(xyz0), n_mcs, _ptr(e), _ptr(m),
                                          _ptr(out)), "plain_metropolis")
    return e, m, out


# ---- the chain -----------------------------------------------------------------------
class Chain:
    """One oracle lattice: init, switch, colour, sweep, observables."""

    def __init__(self, params):
        self.params = params
        h = C.c_void_p()
        _check(lib().sco_ref_init(C.byref(params), C.byref(h)), "init")
        self._h = h
        self.N = params.Lx * params.Ly

    def close(self):
        if self._h:
            lib().sco_ref_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def switch(self):
        _check(lib().sco_ref_switch(self._h), "switch")

    def switch_epoch(self, epoch):
        _check(lib().sco_ref_switch_epoch(self._h, epoch), "switch_epoch")

    def colour(self):
        n = C.c_int32(0)
        _check(lib().sco_ref_colour(self._h, C.byref(n)), "colour")
        return n.value

    def sweep(self, n=1):
        _check(lib().sco_ref_sweep(self._h, n), "sweep")

    def run_series(self, n):
        e = np.zeros(n)
        m = np.zeros(n)
        _check(lib().sco_ref_run_series(self._h, n, _ptr(e), _ptr(m)), "run_series")
        return e, m

    def observables(self, full=False):
        o = Obs()
        _check(lib().sco_ref_observables(self._h, C.byref(o), int(full)), "observables")
        return o.as_dict()

    def spins(self):
        a = np.zeros(3 * self.N)
        _check(lib().sco_ref_get_spins(self._h, _ptr(a)), "get_spins")
        return a

    def set_spins(self, xyz):
        a = np.ascontiguousarray(xyz, np.float64)
        assert a.size == 3 * self.N
        _check(lib().sco_ref_set_spins(self._h, _ptr(a)), "set_spins")

    def graph(self):
        nnz = lib().sco_ref_n_entries(self._h)
        rp = np.zeros(self.N + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.uint32)
        _check(lib().sco_ref_get_graph(self._h, _ptr(rp), _ptr(col), None), "get_graph")
        return rp, col[:nnz]

    def colours(self):
        c = np.zeros(self.N, np.int32)
        _check(lib().sco_ref_get_graph(self._h, None, None, _ptr(c)), "get_colours")
        return c

    def edges(self):
        n = lib().sco_ref_n_half_edges(self._h)
        i = np.zeros(max(n, 1), np.int64)
        j = np.zeros(max(n, 1), np.int64)
        m = np.zeros(max(n, 1), np.int64)
        f = np.zeros(max(n, 1), np.int32)
        _check(lib().sco_ref_get_edges(self._h, _ptr(i), _ptr(j), _ptr(m), _ptr(f)), "get_edges")
        return i[:n], j[:n], m[:n], f[:n]

    def classes(self):
        c = self.colours()
        g = int(c.max()) + 1 if self.N else 1
        rp, _ = self.graph()
        delta = int(np.max(np.diff(rp))) if self.N else 0
        perm = np.zeros(self.N, np.int64)
        off = np.zeros(delta + 2, np.int64)
        _check(lib().sco_ref_get_classes(self._h, _ptr(perm), _ptr(off)), "get_classes")
        assert g <= delta + 1
        return perm, off

    def accepts(self):
        a = np.zeros(self.N, np.uint8)
        _check(lib().sco_ref_get_accepts(self._h, _ptr(a)), "get_accepts")
        return a

    def direct_switch(self, epoch):
        s = np.zeros(self.N * self.N, np.uint8)
        _check(lib().sco_ref_direct_switch(self._h, epoch, _ptr(s)), "direct_switch")
        return s.reshape(self.N, self.N)

    def set_temperature(self, T):
        _check(lib().sco_ref_set_temperature(self._h, float(T)), "set_temperature")
        self.params.T = float(T)

    def graph_stats(self, cells_x=1, cells_y=1, n_rbins=64):
        """P_survive per distance shell, P_IPC and Delta R (see sco_ref_graph_stats)."""
        st = GraphStats()
        surv = np.zeros(n_rbins, np.int64)
        pairs = np.zeros(n_rbins, np.int64)
        ps = np.zeros(n_rbins)
        pal = int(self.colours().max()) + 1 if self.N else 1
        rp, _ = self.graph()
        delta = int(np.max(np.diff(rp))) if self.N else 0
        dr = np.zeros(max(pal, delta + 1))
        _check(lib().sco_ref_graph_stats(self._h, cells_x, cells_y, n_rbins, C.byref(st),
                                         _ptr(surv), _ptr(pairs), _ptr(ps), _ptr(dr)),
               "graph_stats")
        out = st.as_dict()
        out.update(survived=surv, pairs=pairs, p_survive=ps, delta_r=dr[:st.palette])
        return out

    @property
    def sweeps_done(self):
        return lib().sco_ref_sweeps_done(self._h)


def u53(w):
    """u = (w >> 11) 2^-53 as used by every decision."""
    return float(int(w) >> 11) * 2.0 ** -53


def ln2():
    return math.log(2.0)
