"""Thin ctypes binding of libbgk (include/bgk.h): argument marshalling only.

Every step of the stage runs in the library's CUDA kernels; this module only
packs descriptors, passes pointers (numpy arrays as host memory, torch CUDA
tensors as device memory) and turns status codes into exceptions.  There is no
CPU fallback: if libbgk.so is missing the first call raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbgk.so")

BGK_OK, BGK_EINVAL, BGK_ENOMEM, BGK_ECUDA, BGK_ENOCONV, BGK_ETIMEOUT, BGK_ENOTSUP = range(7)
BGK_FP64, BGK_MIXED = 0, 1
BGK_FACE_DIRICHLET, BGK_FACE_SPECULAR, BGK_FACE_DIFFUSE, BGK_FACE_CLOSED = 0, 1, 2, 3
STATUS_NAMES = {0: "BGK_OK", 1: "BGK_EINVAL", 2: "BGK_ENOMEM", 3: "BGK_ECUDA",
                4: "BGK_ENOCONV", 5: "BGK_ETIMEOUT", 6: "BGK_ENOTSUP"}

c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p


class MeshDesc(ctypes.Structure):
    _fields_ = [("n", c_int * 3), ("lo", c_double * 3), ("hi", c_double * 3),
                ("periodic", c_int * 3), ("order", c_int), ("bc_state", (c_double * 5) * 6),
                ("face_type", c_int * 6), ("node_xyz", c_void_p)]


class VGridDesc(ctypes.Structure):
    _fields_ = [("n", c_int * 3), ("lo", c_double * 3), ("hi", c_double * 3)]


class GasDesc(ctypes.Structure):
    _fields_ = [("delta", c_double), ("Pr", c_double), ("mu_ref", c_double),
                ("theta_ref", c_double), ("theta_S", c_double)]


# name -> (restype, argtypes) for every entry point of include/bgk.h
SIGNATURES = {
    "bgk_create": (c_int, [ctypes.POINTER(c_void_p), ctypes.POINTER(MeshDesc),
                           ctypes.POINTER(VGridDesc), ctypes.POINTER(GasDesc), c_int, c_void_p]),
    "bgk_destroy": (c_int, [c_void_p]),
    "bgk_sizes": (c_int, [c_void_p] + [ctypes.POINTER(c_int)] * 4),
    "bgk_node_coords": (c_int, [c_void_p, c_void_p, c_int]),
    "bgk_set_es_tensor": (c_int, [c_void_p, c_int]),
    "bgk_curved_metrics": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "bgk_fr_tables": (c_int, [c_int, c_void_p, c_void_p]),
    "bgk_set_state": (c_int, [c_void_p, c_void_p, c_int]),
    "bgk_get_state": (c_int, [c_void_p, c_void_p, c_int]),
    "bgk_set_maxwellian": (c_int, [c_void_p, c_void_p, c_int]),
    "bgk_set_newton": (c_int, [c_void_p, c_double, c_int]),
    "bgk_set_qprime_engine": (c_int, [c_void_p, c_int]),
    "bgk_set_stage_kernel": (c_int, [c_void_p, c_int, c_int]),
    "bgk_test_ring_stall": (c_int, [c_void_p, c_int, c_double]),
    "bgk_set_velocity_blocks": (c_int, [c_void_p, c_int]),
    "bgk_get_velocity_blocks": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "bgk_set_graphs": (c_int, [c_void_p, c_int]),
    "bgk_tune_stage": (c_int, [c_void_p, c_double, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                               ctypes.POINTER(c_double)]),
    "bgk_rhs": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "bgk_step": (c_int, [c_void_p, c_double, c_int]),
    "bgk_stage": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_double, c_double]),
    "bgk_moments": (c_int, [c_void_p, c_void_p, c_int]),
    "bgk_macro": (c_int, [c_void_p, c_void_p, c_int]),
    "bgk_moments_noalloc": (c_int, [ctypes.POINTER(VGridDesc), c_void_p, c_int, c_int, c_void_p,
                                    c_void_p]),
    "bgk_qprime": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int]),
    "bgk_totals": (c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "bgk_stats": (c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int),
                          ctypes.POINTER(c_double)]),
    "bgk_set_guess": (c_int, [c_void_p, c_int, c_int]),
    "bgk_mlp_log": (c_int, [c_void_p, c_int, ctypes.c_longlong]),
    "bgk_mlp_log_read": (c_int, [c_void_p, c_void_p, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
    "bgk_mlp_train": (c_int, [c_void_p, c_int, c_int, ctypes.c_float, ctypes.c_ulonglong, c_int,
                              ctypes.POINTER(c_double)]),
    "bgk_mlp_weights": (c_int, [c_void_p, c_void_p, c_int]),
    "bgk_mlp_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, ctypes.POINTER(c_double),
                             c_void_p]),
    "bgk_mlp_stats": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_ulonglong)]),
    "bgk_profile": (c_int, [c_void_p, c_int]),
    "bgk_profile_read": (c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "bgk_probe_peak": (c_int, [c_int, ctypes.POINTER(c_double)]),
    "bgk_probe_tc": (c_int, [ctypes.c_longlong, ctypes.POINTER(c_double)]),
    "bgk_step_host": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int]),
    "bgk_step_host_sync": (c_int, [c_void_p]),
    "bgk_create_shard": (c_int, [ctypes.POINTER(c_void_p), c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int,
                                 c_int]),
    "bgk_shard_partials": (c_int, [c_void_p, c_void_p]),
    "bgk_shard_stage": (c_int, [c_void_p, c_void_p, c_int, c_double]),
    "bgk_mlp_infer": (c_int, [c_void_p, c_void_p, ctypes.c_longlong, c_void_p, c_int]),
    "bgk_last_error": (ctypes.c_char_p, [c_void_p]),
}

KERNEL_KINDS = ("moments", "qprime", "stage", "other", "wall")
MLP_NPARAM, MLP_NNORM, MLP_LOG_STRIDE = 5125, 28, 14
MLP_OUT = 5
MLP_SHAPES = ((9, 64), (64,), (64, 64), (64,), (64, 5), (5,))
PROBE_KINDS = {"fp64_fma": 0, "fp32_fma": 1, "fp64_exp": 2, "fp32_exp2": 3}


def probe_peak(kind):
    """Measured device throughput: flop/s for *_fma, calls/s for *_exp*."""
    lib = load()
    v = c_double()
    st = lib.bgk_probe_peak(PROBE_KINDS[kind], ctypes.byref(v))
    if st != BGK_OK:
        raise BGKError(st, "probe %s failed" % kind)
    return v.value


def probe_tc(n_panels):
    """bgk_probe_tc: the p = 3 FR element operator streamed through tcgen05 MMAs.
    Returns a dict: flops, dof_per_s, bytes_per_s, max_rel_err, bias, ms."""
    lib = load()
    out = (c_double * 6)()
    st = lib.bgk_probe_tc(int(n_panels), out)
    if st != BGK_OK:
        raise BGKError(st, "bgk_probe_tc failed")
    keys = ("flops", "dof_per_s", "bytes_per_s", "max_rel_err", "bias", "ms")
    return dict(zip(keys, list(out)))


_lib = None


def load(path=LIB_PATH):
    """Load libbgk.so (raises if it is not built) and declare every signature."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libbgk.so is not built (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        _lib = lib
    return _lib


class BGKError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _ptr(x):
    """(pointer, on_device) of a numpy array (host) or torch tensor (device if CUDA)."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return c_void_p(x.ctypes.data), 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return c_void_p(x.data_ptr()), 1 if x.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor")


def _stream_handle(stream):
    if stream is None:
        return None
    return c_void_p(getattr(stream, "cuda_stream", stream))


def descriptors(wl, node_xyz=None):
    """(MeshDesc, VGridDesc, GasDesc) of a workload definition.  node_xyz: the
    solution-node coordinates [Ne, Ns, 3] of a curvilinear mesh (float64,
    C-contiguous; the caller keeps it alive while the descriptor is used)."""
    m = MeshDesc()
    for d in range(3):
        m.n[d], m.lo[d], m.hi[d] = wl.mesh_n[d], wl.mesh_lo[d], wl.mesh_hi[d]
        m.periodic[d] = 1 if wl.periodic[d] else 0
    m.order = wl.p
    for (d, side), (rho, U, theta) in wl.dirichlet.items():
        row = m.bc_state[2 * d + (1 if side > 0 else 0)]
        row[0], row[1], row[2], row[3], row[4] = rho, U[0], U[1], U[2], theta
    for d, side in getattr(wl, "specular", ()):
        m.face_type[2 * d + (1 if side > 0 else 0)] = BGK_FACE_SPECULAR
    for (d, side), (U_w, theta_w) in getattr(wl, "diffuse", {}).items():
        f = 2 * d + (1 if side > 0 else 0)
        m.face_type[f] = BGK_FACE_DIFFUSE
        row = m.bc_state[f]
        row[0], row[1], row[2], row[3], row[4] = 1.0, U_w[0], U_w[1], U_w[2], theta_w
    for d, side in getattr(wl, "closed", ()):
        m.face_type[2 * d + (1 if side > 0 else 0)] = BGK_FACE_CLOSED
    if node_xyz is not None:
        m.node_xyz = node_xyz.ctypes.data
    v = VGridDesc()
    for d in range(3):
        v.n[d], v.lo[d], v.hi[d] = wl.vel_n[d], wl.vel_lo[d], wl.vel_hi[d]
    g = GasDesc(wl.delta, wl.Pr, wl.mu_ref, wl.theta_ref, wl.theta_S)
    return m, v, g


def fr_tables(order):
    """bgk_fr_tables: the library's FP64 FR operators and the FP32 tables of the
    curvilinear mixed stage, as dicts of numpy arrays (host only)."""
    lib = load()
    q = order + 1
    fr = np.empty(6 * q + q * q)
    c32 = np.empty(q * q + 5 * q, dtype=np.float32)
    st = lib.bgk_fr_tables(order, fr.ctypes.data, c32.ctypes.data)
    if st != BGK_OK:
        raise BGKError(st, "bgk_fr_tables failed")
    names = [("xi", q), ("w", q), ("D", q * q), ("lm", q), ("lp", q), ("dgL", q), ("dgR", q)]
    out, o = {}, 0
    for n, k in names:
        out[n] = fr[o:o + k].copy()
        o += k
    out["D"] = out["D"].reshape(q, q)
    c, o = {}, 0
    for n, k in [("D", q * q), ("lp", q), ("lm", q), ("dgL", q), ("dgR", q), ("def", q)]:
        c[n] = c32[o:o + k].copy()
        o += k
    c["D"] = c["D"].reshape(q, q)
    return out, c


def curved_metrics(wl, node_xyz):
    """bgk_curved_metrics: (S[P, 3, 3] with S[p, d] = S^d, J[P], fvec[Ne, 6, q*q, 3])
    of a curvilinear workload's node coordinates (host only)."""
    lib = load()
    x = np.ascontiguousarray(node_xyz, dtype=np.float64)
    m, _, _ = descriptors(wl, x)
    P = x.shape[0] * x.shape[1]
    q = wl.p + 1
    S = np.empty((P, 3, 3))
    J = np.empty(P)
    fv = np.empty((x.shape[0], 6, q * q, 3))
    st = lib.bgk_curved_metrics(ctypes.byref(m), S.ctypes.data, J.ctypes.data, fv.ctypes.data)
    if st != BGK_OK:
        raise BGKError(st, "bgk_curved_metrics failed")
    return S, J, fv


def _require_cuda_f64(name, t, n):
    """A CUDA float64 contiguous tensor of at least n elements, else ValueError
    (before any library call: the kernels would read or write past it)."""
    if not (hasattr(t, "is_cuda") and hasattr(t, "dtype")):
        raise ValueError("%s must be a CUDA torch tensor, got %s" % (name, type(t).__name__))
    import torch
    if not t.is_cuda:
        raise ValueError("%s must be in device memory" % name)
    if t.dtype != torch.float64:
        raise ValueError("%s must be float64, got %s" % (name, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() < n:
        raise ValueError("%s holds %d elements, the call needs %d" % (name, t.numel(), n))


def moments_noalloc(vgrid, f, n_comp, n_points, m, stream=None):
    """bgk_moments_noalloc: raw moments of a device state into a device output
    without any device allocation by the library (see include/bgk.h).
    vgrid: VGridDesc; f: CUDA tensor [n_comp, N_u, n_points] float64;
    m: CUDA tensor [n_points, 11] float64.  Wrong device, dtype or size
    raises ValueError before the library is called."""
    n_vel = int(vgrid.n[0]) * int(vgrid.n[1]) * int(vgrid.n[2])
    if n_comp not in (1, 2) or n_points <= 0 or n_vel <= 0:
        raise ValueError("n_comp must be 1 or 2 and n_points, N_u positive")
    _require_cuda_f64("f", f, n_comp * n_vel * n_points)
    _require_cuda_f64("m", m, n_points * 11)
    lib = load()
    st = lib.bgk_moments_noalloc(ctypes.byref(vgrid), _ptr(f)[0], n_comp, n_points, _ptr(m)[0],
                                 _stream_handle(stream))
    if st != BGK_OK:
        raise BGKError(st, "bgk_moments_noalloc failed")


class Solver:
    """One libbgk context.  Methods carry the C entry points' names."""

    def __init__(self, wl, precision=BGK_FP64, stream=None, shard=None):
        """shard=(slab_lo, slab_hi): a velocity shard holding the third-axis
        velocity planes [slab_lo, slab_hi) of the workload's grid
        (bgk_create_shard); None: every velocity (bgk_create)."""
        self.lib = load()
        self.wl = wl
        self.precision = precision
        self.shard = tuple(shard) if shard is not None else None
        self._h = c_void_p()
        self._xyz = None
        if getattr(wl, "mapping", None) is not None:
            from . import workloads
            self._xyz = np.ascontiguousarray(workloads.node_positions(wl), dtype=np.float64)
        m, v, g = descriptors(wl, self._xyz)
        if self.shard is None:
            st = self.lib.bgk_create(ctypes.byref(self._h), ctypes.byref(m), ctypes.byref(v),
                                     ctypes.byref(g), precision, _stream_handle(stream))
        else:
            st = self.lib.bgk_create_shard(ctypes.byref(self._h), ctypes.byref(m), ctypes.byref(v),
                                           ctypes.byref(g), precision, _stream_handle(stream),
                                           int(self.shard[0]), int(self.shard[1]))
        if st != BGK_OK:
            msg = self.lib.bgk_last_error(self._h).decode() if self._h else ""
            if self._h:
                self.lib.bgk_destroy(self._h)
                self._h = c_void_p()
            raise BGKError(st, msg)
        ne, ns, nu, nc = c_int(), c_int(), c_int(), c_int()
        self._check(self.lib.bgk_sizes(self._h, ctypes.byref(ne), ctypes.byref(ns),
                                       ctypes.byref(nu), ctypes.byref(nc)))
        self.n_elem, self.n_sol, self.n_vel, self.n_comp = ne.value, ns.value, nu.value, nc.value
        self.dtype = np.float64 if precision == BGK_FP64 else np.float32
        if getattr(wl, "es_tensor", False):
            self.set_es_tensor(True)

    @property
    def shape(self):
        return (self.n_comp, self.n_vel, self.n_elem, self.n_sol)

    @property
    def n_points(self):
        return self.n_elem * self.n_sol

    def _check(self, st):
        if st != BGK_OK:
            raise BGKError(st, self.lib.bgk_last_error(self._h).decode())

    def destroy(self):
        if self._h:
            self.lib.bgk_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    # -- entry points ------------------------------------------------------
    def node_coords(self):
        x = np.empty((self.n_elem, self.n_sol, 3))
        p, dev = _ptr(x)
        self._check(self.lib.bgk_node_coords(self._h, p, dev))
        return x

    def set_es_tensor(self, enable=True):
        self._check(self.lib.bgk_set_es_tensor(self._h, 1 if enable else 0))

    def set_state(self, f):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=self.dtype)
        if tuple(f.shape) != self.shape:
            raise ValueError("state shape %s, expected %s" % (tuple(f.shape), self.shape))
        p, dev = _ptr(f)
        self._check(self.lib.bgk_set_state(self._h, p, dev))

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype)
        p, dev = _ptr(out)
        self._check(self.lib.bgk_get_state(self._h, p, dev))
        return out

    def set_maxwellian(self, q):
        if isinstance(q, np.ndarray):
            q = np.ascontiguousarray(q, dtype=np.float64).reshape(self.n_points, 5)
        p, dev = _ptr(q)
        self._check(self.lib.bgk_set_maxwellian(self._h, p, dev))

    def set_newton(self, tol=1e-13, max_iter=50):
        self._check(self.lib.bgk_set_newton(self._h, tol, max_iter))

    def set_qprime_engine(self, fp32_sums):
        self._check(self.lib.bgk_set_qprime_engine(self._h, 1 if fp32_sums else 0))

    def set_velocity_blocks(self, n):
        self._check(self.lib.bgk_set_velocity_blocks(self._h, int(n)))

    def velocity_blocks(self):
        """(number of velocity blocks, velocities per block, most blocks accepted)."""
        n, per, mx = c_int(), c_int(), c_int()
        self._check(self.lib.bgk_get_velocity_blocks(self._h, ctypes.byref(n), ctypes.byref(per), ctypes.byref(mx)))
        return n.value, per.value, mx.value

    def test_ring_stall(self, after, wait_seconds=0.0):
        """Test entry: the copy rings deliver only `after` velocities per block
        (0 restores), the bounded waits give up after wait_seconds."""
        self._check(self.lib.bgk_test_ring_stall(self._h, int(after), float(wait_seconds)))

    STAGE_KERNELS = {"auto": 0, "plain": 1, "async": 2, "line": 3, "line_wide": 4, "half": 5, "half_wide": 6}

    def set_stage_kernel(self, variant="auto", depth=6):
        """Mixed-form stage kernel: "auto", "plain", "async", "line", "line_wide", "half" or
        "half_wide" (all but the first two on a bulk-copy ring of `depth` stages)."""
        self._check(self.lib.bgk_set_stage_kernel(self._h, self.STAGE_KERNELS[variant], int(depth)))

    def set_graphs(self, enable=True):
        """bgk_step as CUDA-graph replays (captured per buffer parity)."""
        self._check(self.lib.bgk_set_graphs(self._h, 1 if enable else 0))

    def tune_stage(self, dt, reps=3):
        """Time the stage kernel candidates on this problem, keep the fastest;
        returns (variant name, depth, ms per stage)."""
        v, d, ms = c_int(), c_int(), c_double()
        self._check(self.lib.bgk_tune_stage(self._h, dt, int(reps), ctypes.byref(v), ctypes.byref(d),
                                            ctypes.byref(ms)))
        names = {b: a for a, b in self.STAGE_KERNELS.items()}
        return names[v.value], d.value, ms.value

    def rhs(self, f, out=None):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=self.dtype)
            out = np.empty(self.shape, dtype=self.dtype) if out is None else out
        pf, dev = _ptr(f)
        po, dev2 = _ptr(out)
        if dev != dev2:
            raise ValueError("input and output must both be host or both be device")
        self._check(self.lib.bgk_rhs(self._h, pf, po, dev))
        return out

    def step(self, dt, n_steps=1):
        """Returns the status code (BGK_OK, or BGK_ENOCONV if a solve did not
        converge); other failures raise."""
        st = self.lib.bgk_step(self._h, dt, n_steps)
        if st not in (BGK_OK, BGK_ENOCONV):
            self._check(st)
        return st

    def stage(self, f_n, f_in, f_out, a, b, c):
        pn = _ptr(f_n)[0] if f_n is not None else None
        self._check(self.lib.bgk_stage(self._h, pn, _ptr(f_in)[0], _ptr(f_out)[0], a, b, c))

    def moments(self, out=None):
        out = np.empty((self.n_points, 11)) if out is None else out
        p, dev = _ptr(out)
        self._check(self.lib.bgk_moments(self._h, p, dev))
        return out

    MACRO_FIELDS = ("rho", "U1", "U2", "U3", "theta", "p", "mach", "lambda", "grad_rho", "kn_gll")

    def macro(self, out=None):
        """[n_points, 10] macroscopic fields (MACRO_FIELDS), incl. Kn_GLL."""
        out = np.empty((self.n_points, 10)) if out is None else out
        p, dev = _ptr(out)
        self._check(self.lib.bgk_macro(self._h, p, dev))
        return out

    def qprime(self, m):
        m = np.ascontiguousarray(m, dtype=np.float64)
        n = m.shape[0]
        qp = np.empty((n, 5))
        it = np.empty(n, dtype=np.int32)
        st = self.lib.bgk_qprime(self._h, _ptr(m)[0], n, _ptr(qp)[0], _ptr(it)[0], 0)
        if st not in (BGK_OK, BGK_ENOCONV):
            self._check(st)
        return qp, it, st

    def totals(self):
        t = (c_double * 5)()
        self._check(self.lib.bgk_totals(self._h, t, None))
        return np.array(list(t))

    def entropy(self):
        """bgk_totals' entropy output: sum W J sum_k w F ln F of the stored F (NaN if some F <= 0)."""
        t = (c_double * 5)()
        h = c_double()
        self._check(self.lib.bgk_totals(self._h, t, ctypes.byref(h)))
        return h.value

    def stats(self):
        mean, mx, res = c_double(), c_int(), c_double()
        self._check(self.lib.bgk_stats(self._h, ctypes.byref(mean), ctypes.byref(mx),
                                       ctypes.byref(res)))
        return mean.value, mx.value, res.value

    # -- learned Q' guess ----------------------------------------------------
    def set_guess(self, mode, bf16=True):
        self._check(self.lib.bgk_set_guess(self._h, int(mode), 1 if bf16 else 0))

    def mlp_log(self, enable=True, max_pairs=1 << 20):
        self._check(self.lib.bgk_mlp_log(self._h, 1 if enable else 0, int(max_pairs)))

    def mlp_log_read(self, max_pairs=1 << 20):
        out = np.empty((max_pairs, MLP_LOG_STRIDE), dtype=np.float32)
        n = ctypes.c_longlong()
        self._check(self.lib.bgk_mlp_log_read(self._h, _ptr(out)[0], max_pairs, ctypes.byref(n)))
        return out[:n.value]

    def mlp_train(self, epochs=20, batch=4096, lr=1e-3, seed=0, bf16=True):
        loss = c_double()
        self._check(self.lib.bgk_mlp_train(self._h, epochs, batch, lr, seed, 1 if bf16 else 0,
                                           ctypes.byref(loss)))
        return loss.value

    def mlp_weights(self, load=None):
        """Return (params list, norm) or load them (params list of arrays, norm[28])."""
        buf = np.empty(MLP_NPARAM + MLP_NNORM, dtype=np.float32)
        if load is None:
            self._check(self.lib.bgk_mlp_weights(self._h, _ptr(buf)[0], 0))
            params, off = [], 0
            for shp in MLP_SHAPES:
                n = int(np.prod(shp))
                params.append(buf[off:off + n].reshape(shp).copy())
                off += n
            return params, buf[MLP_NPARAM:].copy()
        params, norm = load
        buf[:MLP_NPARAM] = np.concatenate([np.asarray(p, dtype=np.float32).ravel() for p in params])
        buf[MLP_NPARAM:] = np.asarray(norm, dtype=np.float32)
        self._check(self.lib.bgk_mlp_weights(self._h, _ptr(buf)[0], 1))

    def mlp_grad(self, x, t, bf16=True):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.empty(MLP_NPARAM, dtype=np.float32)
        loss = c_double()
        self._check(self.lib.bgk_mlp_grad(self._h, _ptr(x)[0], _ptr(t)[0], x.shape[0],
                                          1 if bf16 else 0, ctypes.byref(loss), _ptr(g)[0]))
        grads, off = [], 0
        for shp in MLP_SHAPES:
            n = int(np.prod(shp))
            grads.append(g[off:off + n].reshape(shp).astype(np.float64))
            off += n
        return loss.value, grads

    def step_host(self, f_in, f_out, dt, n_steps=1):
        """bgk_step_host: enqueue f_in (host) -> n_steps -> f_out (host); returns
        at once.  Keep both buffers alive until step_host_sync()."""
        pi, din = _ptr(f_in)
        po, dout = _ptr(f_out)
        if din or dout:
            raise ValueError("step_host takes host buffers (pinned for the full copy rate)")
        for t in (f_in, f_out):
            if tuple(t.shape) != self.shape:
                raise ValueError("state shape %s, expected %s" % (tuple(t.shape), self.shape))
            if np.dtype(str(t.dtype).replace("torch.", "")) != np.dtype(self.dtype):
                raise ValueError("state dtype %s, expected %s" % (t.dtype, np.dtype(self.dtype)))
        self._check(self.lib.bgk_step_host(self._h, pi, po, float(dt), int(n_steps)))

    def step_host_sync(self):
        """bgk_step_host_sync: wait for every step_host call; returns the status."""
        st = self.lib.bgk_step_host_sync(self._h)
        if st not in (BGK_OK, BGK_ENOCONV):
            self._check(st)
        return st

    # -- velocity shards -------------------------------------------------------
    def shard_partials(self, m):
        """bgk_shard_partials into the device tensor m[11, n_points] (float64)."""
        if not (getattr(m, "is_cuda", False) and m.dtype.is_floating_point and m.element_size() == 8
                and m.is_contiguous() and m.numel() >= 11 * self.n_points):
            raise ValueError("m must be a contiguous CUDA float64 tensor of 11 x n_points")
        self._check(self.lib.bgk_shard_partials(self._h, _ptr(m)[0]))

    def shard_stage(self, m, stage, dt):
        """bgk_shard_stage from the summed moments m[11, n_points] (device)."""
        if not (getattr(m, "is_cuda", False) and m.element_size() == 8 and m.is_contiguous()
                and m.numel() >= 11 * self.n_points):
            raise ValueError("m must be a contiguous CUDA float64 tensor of 11 x n_points")
        st = self.lib.bgk_shard_stage(self._h, _ptr(m)[0], int(stage), float(dt))
        if st not in (BGK_OK, BGK_ENOCONV):
            self._check(st)
        return st

    def mlp_infer(self, x, out=None):
        """bgk_mlp_infer: delta[n, 5] of raw features x[n, 9] (numpy or CUDA tensors)."""
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float32)
            out = np.empty((x.shape[0], MLP_OUT), dtype=np.float32) if out is None else out
        n = x.shape[0]
        px, dev = _ptr(x)
        po, dev_o = _ptr(out)
        if dev != dev_o:
            raise ValueError("x and out must both be host or both be device memory")
        self._check(self.lib.bgk_mlp_infer(self._h, px, n, po, dev))
        return out

    def mlp_stats(self):
        n = ctypes.c_ulonglong()
        self._check(self.lib.bgk_mlp_stats(self._h, ctypes.byref(n)))
        return n.value

    def profile(self, enable=True):
        self._check(self.lib.bgk_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """{kind: (ms, launches)} since the last profile(True)."""
        ms = (c_double * len(KERNEL_KINDS))()
        n = (ctypes.c_longlong * len(KERNEL_KINDS))()
        self._check(self.lib.bgk_profile_read(self._h, ms, n))
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_KINDS)}

    def last_error(self):
        return self.lib.bgk_last_error(self._h).decode()
