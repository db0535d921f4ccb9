"""GB300 library for the per-sweep hot path of the parallelized stochastic cutoff (SCO)
method (Endo, Toga and Sasaki, arXiv:1503.03295).

This module only marshals arguments to the C ABI of ``lib/libsco.so`` (declared in
``include/sco.h``); every step of the path runs in the library's CUDA kernels.  There is
no fallback: importing works anywhere, but creating a :class:`Lattice` without a usable
CUDA device, or without the built library, raises.
"""
import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libsco.so")

SCO_OK, SCO_EINVAL, SCO_ENOMEM, SCO_ECUDA, SCO_ETIMEOUT, SCO_ESTATE, SCO_EGUARD, SCO_ECAPACITY = range(8)
KW_STATIC_MAX_VERTICES = 1 << 20
FP64, FP32_GUARDED = 0, 1
EXCH_ONLY = 0x80000000


class ScoError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, strerror(status), status))


class Params(C.Structure):
    _fields_ = [("Lx", C.c_int32), ("Ly", C.c_int32), ("J", C.c_double), ("D", C.c_double),
                ("T", C.c_double), ("seed", C.c_uint64), ("n_sw", C.c_int32),
                ("precision", C.c_int32), ("colour_variant", C.c_int32), ("replica", C.c_int32)]


class BatchTuning(C.Structure):
    _fields_ = [("steps_per_graph", C.c_int32), ("sweep_blocks_per_sm", C.c_int32),
                ("kw_blocks_per_sm", C.c_int32), ("use_graph", C.c_int32),
                ("kw_schedule", C.c_int32), ("kw_low", C.c_int32),
                ("kw_low_group", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Obs(C.Structure):
    _fields_ = [("e_switched", C.c_double), ("e_exchange", C.c_double), ("e_full", C.c_double),
                ("mx", C.c_double), ("my", C.c_double), ("mz", C.c_double),
                ("m_abs", C.c_double), ("m_phi", C.c_double), ("n_edges", C.c_int64),
                ("max_degree", C.c_int32), ("n_colours", C.c_int32), ("kw_rounds", C.c_int32),
                ("max_degree_dipolar", C.c_int32), ("sweeps_done", C.c_int64),
                ("guard_hits_fp64", C.c_int64), ("guard_hits_fp32", C.c_int64),
                ("kernel_launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GraphStats(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("n_cross", C.c_int64), ("p_ipc", C.c_double),
                ("delta_r_mean", C.c_double), ("delta_r_max", C.c_double),
                ("delta_r_weighted", C.c_double), ("n_cells", C.c_int32), ("palette", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load():
    """Load lib/libsco.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsco.so is not built; run paper_1503_03295_gb300._build.build() "
                           "or __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, st = C.c_void_p, C.c_int
    sig = {
        "sco_init": ([C.POINTER(Params), vp, C.POINTER(vp)], st),
        "sco_destroy": ([vp], None),
        "sco_switch": ([vp], st),
        "sco_colour": ([vp, C.POINTER(C.c_int32)], st),
        "sco_sweep": ([vp, C.c_int32], st),
        "sco_observables": ([vp, C.POINTER(Obs), C.c_int32], st),
        "sco_get_spins": ([vp, vp, C.c_int32], st),
        "sco_set_spins": ([vp, vp, C.c_int32], st),
        "sco_get_sizes": ([vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                           C.POINTER(C.c_int32)], st),
        "sco_get_graph": ([vp, vp, vp, vp], st),
        "sco_get_classes": ([vp, vp, vp], st),
        "sco_get_accepts": ([vp, vp], st),
        "sco_get_table": ([vp, C.POINTER(C.c_int64), vp, vp, vp, vp], st),
        "sco_get_state": ([vp, vp, C.POINTER(C.c_size_t)], st),
        "sco_set_state": ([vp, vp, C.c_size_t], st),
        "sco_set_timing": ([vp, C.c_int32], st),
        "sco_get_timing": ([vp, vp, vp], st),
        "sco_sync": ([vp], st),
        "sco_set_wait_limit": ([vp, C.c_uint64], st),
        "sco_set_temperature": ([vp, C.c_double], st),
        "sco_get_graph_stats": ([vp, C.c_int32, C.c_int32, C.c_int32, C.POINTER(GraphStats),
                                 vp, vp, vp, vp], st),
        "sco_batch_set_wait_limit": ([vp, C.c_uint64], st),
        "sco_batch_set_temperature": ([vp, C.c_int32, C.c_double], st),
        "sco_kw_colour_static": ([vp, vp, C.c_int64, C.c_int32, vp, C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int32), vp], st),
        "sco_strerror": ([C.c_int], C.c_char_p),
        "sco_batch_init": ([vp, C.c_int32, vp, C.POINTER(vp)], st),
        "sco_batch_destroy": ([vp], None),
        "sco_batch_run": ([vp, C.c_int32], st),
        "sco_batch_autotune": ([vp, C.c_int32, C.POINTER(BatchTuning)], st),
        "sco_batch_set_tuning": ([vp, C.POINTER(BatchTuning)], st),
        "sco_batch_get_tuning": ([vp, C.POINTER(BatchTuning)], st),
        "sco_batch_observables": ([vp, C.c_int32, C.POINTER(Obs), C.c_int32], st),
        "sco_batch_get_spins": ([vp, C.c_int32, vp, C.c_int32], st),
        "sco_batch_set_spins": ([vp, C.c_int32, vp, C.c_int32], st),
        "sco_batch_get_sizes": ([vp, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int32), C.POINTER(C.c_int32)], st),
        "sco_batch_get_graph": ([vp, C.c_int32, vp, vp, vp], st),
        "sco_batch_get_accepts": ([vp, C.c_int32, vp], st),
        "sco_batch_info": ([vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                            C.POINTER(C.c_int64), C.POINTER(C.c_int32)], st),
        "sco_batch_sync": ([vp], st),
        "sco_selftest_expm1_deg": ([C.c_int64, C.c_uint64, C.c_int32, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)], st),
        "sco_selftest_log": ([C.c_int64, C.c_uint64, C.POINTER(C.c_double),
                              C.POINTER(C.c_double)], st),
        "sco_selftest_expm1": ([C.c_int64, C.c_uint64, C.POINTER(C.c_double),
                                C.POINTER(C.c_double)], st),
        "sco_probe_fp64": ([C.c_int64, vp], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def strerror(status):
    try:
        return load().sco_strerror(int(status)).decode()
    except Exception:
        return "status %d" % status


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _check(status, what):
    if status != SCO_OK:
        raise ScoError(status, what)


def kw_colour_static(row_ptr_dev, col_dev, n, colour_dev, variant=0, stream=None):
    """Allocation-free colouring of a caller's CSR graph held in device memory (raw device
    pointers as ints).  Returns (max_degree, t_R).  See sco_kw_colour_static in sco.h."""
    d, r = C.c_int32(0), C.c_int32(0)
    _check(load().sco_kw_colour_static(C.c_void_p(row_ptr_dev), C.c_void_p(col_dev), int(n),
                                       int(variant), C.c_void_p(colour_dev), C.byref(d),
                                       C.byref(r), C.c_void_p(stream or 0)),
           "sco_kw_colour_static")
    return d.value, r.value


def selftest_expm1(n=1 << 24, seed=1, degree=8):
    """Largest relative error of the library's expm1 (x <= 0.35; polynomial degree 8 or 6)
    against double-double and against CUDA's expm1 (see sco_selftest_expm1_deg)."""
    a, b = C.c_double(), C.c_double()
    _check(load().sco_selftest_expm1_deg(int(n), int(seed), int(degree), C.byref(a), C.byref(b)),
           "sco_selftest_expm1_deg")
    return a.value, b.value


def selftest_log(n=1 << 24, seed=1):
    """Largest relative error of the library's log (0 < x <= 1) against double-double and
    against CUDA's log (see sco_selftest_log)."""
    a, b = C.c_double(), C.c_double()
    _check(load().sco_selftest_log(int(n), int(seed), C.byref(a), C.byref(b)), "sco_selftest_log")
    return a.value, b.value


def probe_fp64(iters=8192):
    """Measured FP64 throughput of the current device (see sco_probe_fp64): FMA lane-operations,
    library expm1 (degree 6) and log evaluations per second."""
    out = np.zeros(3)
    _check(load().sco_probe_fp64(int(iters), _ptr(out)), "sco_probe_fp64")
    return {"dfma_per_s": float(out[0]), "flops": 2.0 * float(out[0]),
            "expm1_per_s": float(out[1]), "log_per_s": float(out[2])}


def make_params(Lx, Ly=None, T=1.0, D=1.0, J=0.0, seed=0, n_sw=1, precision=FP64,
                colour_variant=0, replica=0):
    return Params(Lx, Lx if Ly is None else Ly, J, D, T, seed, n_sw, precision, colour_variant,
                  replica)


class Lattice:
    """One SCO lattice on the GPU (a thin handle on ``sco_ctx``).

    ``stream`` is a CUDA stream handle (int) or None for the legacy default stream, e.g.
    ``torch.cuda.current_stream().cuda_stream``.
    """

    def __init__(self, params=None, stream=None, **kw):
        self.params = params if params is not None else make_params(**kw)
        L = load()
        h = C.c_void_p()
        _check(L.sco_init(C.byref(self.params), C.c_void_p(stream or 0), C.byref(h)), "sco_init")
        self._h = h
        self.N = self.params.Lx * self.params.Ly

    def close(self):
        if getattr(self, "_h", None):
            load().sco_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # ---- the path -------------------------------------------------------------------
    def switch(self):
        _check(load().sco_switch(self._h), "sco_switch")

    def colour(self, count=True):
        n = C.c_int32(0)
        _check(load().sco_colour(self._h, C.byref(n) if count else None), "sco_colour")
        return n.value if count else None

    def sweep(self, n=1):
        _check(load().sco_sweep(self._h, int(n)), "sco_sweep")

    def observables(self, full=False):
        o = Obs()
        _check(load().sco_observables(self._h, C.byref(o), int(bool(full))), "sco_observables")
        return o.as_dict()

    def sync(self):
        _check(load().sco_sync(self._h), "sco_sync")

    def set_wait_limit(self, ns):
        """Bound (ns) of every device-side wait (see sco_set_wait_limit)."""
        _check(load().sco_set_wait_limit(self._h, int(ns)), "sco_set_wait_limit")

    def set_temperature(self, T):
        """New temperature; the next MC step switches again (see sco_set_temperature)."""
        _check(load().sco_set_temperature(self._h, float(T)), "sco_set_temperature")
        self.params.T = float(T)

    def graph_stats(self, cells_x=1, cells_y=1, n_rbins=64):
        """P_survive per distance shell, P_IPC of a cells_x x cells_y split and Delta R per
        colour of the current graph (see sco_get_graph_stats)."""
        _, _, _, g = self.sizes()
        st = GraphStats()
        surv = np.zeros(n_rbins, np.int64)
        pairs = np.zeros(n_rbins, np.int64)
        ps = np.zeros(n_rbins)
        dr = np.zeros(max(g, 1))
        _check(load().sco_get_graph_stats(self._h, int(cells_x), int(cells_y), int(n_rbins),
                                          C.byref(st), _ptr(surv), _ptr(pairs), _ptr(ps),
                                          _ptr(dr)), "sco_get_graph_stats")
        out = st.as_dict()
        out.update(survived=surv, pairs=pairs, p_survive=ps, delta_r=dr[:st.palette])
        return out

    # ---- data -----------------------------------------------------------------------
    def spins(self):
        a = np.empty(3 * self.N)
        _check(load().sco_get_spins(self._h, _ptr(a), 0), "sco_get_spins")
        return a

    def set_spins(self, xyz):
        a = np.ascontiguousarray(xyz, np.float64)
        if a.size != 3 * self.N:
            raise ValueError("expected %d values" % (3 * self.N))
        _check(load().sco_set_spins(self._h, _ptr(a), 0), "sco_set_spins")

    def get_spins_device(self, dev_ptr):
        _check(load().sco_get_spins(self._h, C.c_void_p(dev_ptr), 1), "sco_get_spins")

    def set_spins_device(self, dev_ptr):
        _check(load().sco_set_spins(self._h, C.c_void_p(dev_ptr), 1), "sco_set_spins")

    def sizes(self):
        n, e, d, g = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int32()
        _check(load().sco_get_sizes(self._h, C.byref(n), C.byref(e), C.byref(d), C.byref(g)),
               "sco_get_sizes")
        return n.value, e.value, d.value, g.value

    def graph(self):
        _, nnz, _, _ = self.sizes()
        rp = np.empty(self.N + 1, np.uint32)
        col = np.empty(max(nnz, 1), np.uint32)
        _check(load().sco_get_graph(self._h, _ptr(rp), _ptr(col), None), "sco_get_graph")
        return rp, col[:nnz]

    def colours(self):
        c = np.empty(self.N, np.uint32)
        _check(load().sco_get_graph(self._h, None, None, _ptr(c)), "sco_get_graph")
        return c

    def classes(self):
        _, _, _, g = self.sizes()
        perm = np.empty(self.N, np.uint32)
        off = np.empty(g + 1, np.uint32)
        _check(load().sco_get_classes(self._h, _ptr(perm), _ptr(off)), "sco_get_classes")
        return perm, off

    def accepts(self):
        a = np.empty(self.N, np.uint8)
        _check(load().sco_get_accepts(self._h, _ptr(a)), "sco_get_accepts")
        return a

    def table(self):
        K = C.c_int64()
        _check(load().sco_get_table(self._h, C.byref(K), None, None, None, None), "sco_get_table")
        k = K.value
        dx, dy = np.empty(k, np.int32), np.empty(k, np.int32)
        W, cc = np.empty(k, np.uint64), np.empty(k)
        _check(load().sco_get_table(self._h, C.byref(K), _ptr(dx), _ptr(dy), _ptr(W), _ptr(cc)),
               "sco_get_table")
        return dict(dx=dx, dy=dy, W=W, Dc=cc)

    def get_state(self):
        n = C.c_size_t(0)
        _check(load().sco_get_state(self._h, None, C.byref(n)), "sco_get_state")
        buf = np.empty(n.value, np.uint8)
        _check(load().sco_get_state(self._h, _ptr(buf), C.byref(n)), "sco_get_state")
        return buf.tobytes()

    def set_state(self, blob):
        buf = np.frombuffer(blob, np.uint8).copy()
        _check(load().sco_set_state(self._h, _ptr(buf), buf.size), "sco_set_state")

    def set_timing(self, enable=True):
        _check(load().sco_set_timing(self._h, int(bool(enable))), "sco_set_timing")

    def timing(self):
        ms = np.zeros(3)
        calls = np.zeros(3, np.int64)
        _check(load().sco_get_timing(self._h, _ptr(ms), _ptr(calls)), "sco_get_timing")
        return dict(switch_ms=ms[0], colour_ms=ms[1], sweep_ms=ms[2], switch_calls=int(calls[0]),
                    colour_calls=int(calls[1]), sweep_calls=int(calls[2]))


class Batch:
    """Replicas that advance together (a thin handle on ``sco_batch``): one launch per phase
    over all replicas, runs of steps replayed as CUDA graphs.  ``params`` is a list of
    :class:`Params` (one precision and one n_sw for all).  ``stream`` None lets the batch
    own a stream."""

    def __init__(self, params, stream=None):
        self.params = list(params)
        arr = (Params * len(self.params))(*self.params)
        h = C.c_void_p()
        _check(load().sco_batch_init(arr, len(self.params), C.c_void_p(stream or 0), C.byref(h)),
               "sco_batch_init")
        self._h = h
        self.N = [p.Lx * p.Ly for p in self.params]

    def close(self):
        if getattr(self, "_h", None):
            load().sco_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __len__(self):
        return len(self.params)

    def run(self, n=1):
        _check(load().sco_batch_run(self._h, int(n)), "sco_batch_run")

    def sync(self):
        _check(load().sco_batch_sync(self._h), "sco_batch_sync")

    def set_wait_limit(self, ns):
        _check(load().sco_batch_set_wait_limit(self._h, int(ns)), "sco_batch_set_wait_limit")

    def set_temperature(self, r, T):
        """Replica r's new temperature, between steps t with t mod n_sw = 0 (see
        sco_batch_set_temperature)."""
        _check(load().sco_batch_set_temperature(self._h, int(r), float(T)),
               "sco_batch_set_temperature")
        self.params[r].T = float(T)

    def autotune(self, trial_steps=2):
        t = BatchTuning()
        _check(load().sco_batch_autotune(self._h, int(trial_steps), C.byref(t)),
               "sco_batch_autotune")
        return t.as_dict()

    def set_tuning(self, steps_per_graph=4, sweep_blocks_per_sm=1, kw_blocks_per_sm=1,
                   use_graph=1, kw_schedule=0, kw_low=1, kw_low_group=2048):
        t = BatchTuning(steps_per_graph, sweep_blocks_per_sm, kw_blocks_per_sm, use_graph,
                        kw_schedule, kw_low, kw_low_group)
        _check(load().sco_batch_set_tuning(self._h, C.byref(t)), "sco_batch_set_tuning")

    def tuning(self):
        t = BatchTuning()
        _check(load().sco_batch_get_tuning(self._h, C.byref(t)), "sco_batch_get_tuning")
        return t.as_dict()

    def info(self):
        a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        e = C.c_int32()
        _check(load().sco_batch_info(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d),
                                     C.byref(e)), "sco_batch_info")
        return dict(total_sites=a.value, steps_done=b.value, launches=c.value,
                    graph_launches=d.value, replans=e.value)

    def observables(self, r, full=False):
        o = Obs()
        _check(load().sco_batch_observables(self._h, int(r), C.byref(o), int(bool(full))),
               "sco_batch_observables")
        return o.as_dict()

    def spins(self, r):
        a = np.empty(3 * self.N[r])
        _check(load().sco_batch_get_spins(self._h, int(r), _ptr(a), 0), "sco_batch_get_spins")
        return a

    def set_spins(self, r, xyz):
        a = np.ascontiguousarray(xyz, np.float64)
        if a.size != 3 * self.N[r]:
            raise ValueError("expected %d values" % (3 * self.N[r]))
        _check(load().sco_batch_set_spins(self._h, int(r), _ptr(a), 0), "sco_batch_set_spins")

    def get_spins_device(self, r, dev_ptr):
        _check(load().sco_batch_get_spins(self._h, int(r), C.c_void_p(dev_ptr), 1),
               "sco_batch_get_spins")

    def set_spins_device(self, r, dev_ptr):
        _check(load().sco_batch_set_spins(self._h, int(r), C.c_void_p(dev_ptr), 1),
               "sco_batch_set_spins")

    def sizes(self, r):
        n, e, d, g = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int32()
        _check(load().sco_batch_get_sizes(self._h, int(r), C.byref(n), C.byref(e), C.byref(d),
                                          C.byref(g)), "sco_batch_get_sizes")
        return n.value, e.value, d.value, g.value

    def graph(self, r):
        _, nnz, _, _ = self.sizes(r)
        rp = np.empty(self.N[r] + 1, np.uint32)
        col = np.empty(max(nnz, 1), np.uint32)
        _check(load().sco_batch_get_graph(self._h, int(r), _ptr(rp), _ptr(col), None),
               "sco_batch_get_graph")
        return rp, col[:nnz]

    def colours(self, r):
        c = np.empty(self.N[r], np.uint32)
        _check(load().sco_batch_get_graph(self._h, int(r), None, None, _ptr(c)),
               "sco_batch_get_graph")
        return c

    def accepts(self, r):
        a = np.empty(self.N[r], np.uint8)
        _check(load().sco_batch_get_accepts(self._h, int(r), _ptr(a)), "sco_batch_get_accepts")
        return a


def replica_params(L_list=(64, 128, 256, 512), n_T=16, T_lo=0.2, T_hi=1.5,
                   precision=FP32_GUARDED, **kw):
    """Replica r = n_T a + b: L = L_list[a], T = (T_lo + b (T_hi - T_lo) / (n_T - 1)) D,
    seed r (the batched workload: 4 sizes x 16 temperatures)."""
    out = []
    for a, L in enumerate(L_list):
        for b in range(n_T):
            r = n_T * a + b
            T = T_lo + b * (T_hi - T_lo) / (n_T - 1) if n_T > 1 else T_lo
            out.append(make_params(L, T=T, seed=r, precision=precision, **kw))
    return out
