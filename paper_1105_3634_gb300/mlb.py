"""Thin ctypes binding of the C ABI in include/mlb.h (same names), plus a
small convenience wrapper.  Argument marshalling only: every step of the
method runs in the CUDA kernels of libmlb.so.  There is no fallback: if the
library is missing or cannot load, importing raises.

PyTorch supplies device memory (its caching allocator, through the
``dev_alloc``/``dev_free`` callbacks) and the CUDA stream the context launches
on.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmlb.so")

MLB_Q = 19
MLB_MAX_SPECIES = 4
MLB_DRAG_ONLY = 1
MLB_FORCE_EXPLICIT = 2
MLB_SPLIT_COLLIDE = 4
MLB_MEANFIELD_BF16 = 8
MLB_MEANFIELD_BF16_1PASS = 16

STATUS = {0: "MLB_OK", 1: "MLB_EINVAL", 2: "MLB_ENOMEM", 3: "MLB_ECUDA", 4: "MLB_ENUMERIC",
          5: "MLB_ETIMEOUT", 6: "MLB_ESTATE"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class mlb_lattice_desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("nspecies", ctypes.c_int32), ("wall_axis", ctypes.c_int32), ("flags", ctypes.c_uint32),
        ("wall_u_lo", ctypes.c_double * 3), ("wall_u_hi", ctypes.c_double * 3),
        ("tau", ctypes.c_double), ("kT", ctypes.c_double), ("kappa", ctypes.c_double),
        ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_user", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
    ]


class MLBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_1105_3634_gb300.build.build() "
                          "(the CUDA library is required; there is no CPU path)")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, fp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
    st = ctypes.c_int
    L.mlb_create.argtypes = [ctypes.POINTER(mlb_lattice_desc), ctypes.POINTER(vp)]
    L.mlb_create.restype = st
    L.mlb_set_species.argtypes = [vp, dp, dp]
    L.mlb_set_species.restype = st
    L.mlb_set_interactions.argtypes = [vp, dp, dp]
    L.mlb_set_interactions.restype = st
    L.mlb_set_fields.argtypes = [vp, dp, dp]
    L.mlb_set_fields.restype = st
    L.mlb_set_external_force.argtypes = [vp, dp]
    L.mlb_set_external_force.restype = st
    L.mlb_step.argtypes = [vp, ctypes.c_int64]
    L.mlb_step.restype = st
    L.mlb_set_predictor_sweeps.argtypes = [vp, ctypes.c_int32]
    L.mlb_set_predictor_sweeps.restype = st
    L.mlb_synchronize.argtypes = [vp]
    L.mlb_synchronize.restype = st
    L.mlb_get_moments.argtypes = [vp, dp, dp]
    L.mlb_get_moments.restype = st
    L.mlb_get_acceleration.argtypes = [vp, dp]
    L.mlb_get_acceleration.restype = st
    L.mlb_conservation.argtypes = [vp, dp, dp]
    L.mlb_conservation.restype = st
    L.mlb_get_populations.argtypes = [vp, fp, dp, ctypes.POINTER(ctypes.c_int64)]
    L.mlb_get_populations.restype = st
    L.mlb_set_populations.argtypes = [vp, fp, dp, ctypes.c_int64]
    L.mlb_set_populations.restype = st
    L.mlb_velocity_set.argtypes = [ctypes.POINTER(ctypes.c_int32), dp]
    L.mlb_velocity_set.restype = st
    L.mlb_launches_per_step.argtypes = [vp]
    L.mlb_launches_per_step.restype = ctypes.c_int32
    L.mlb_profile_enable.argtypes = [vp, ctypes.c_int32]
    L.mlb_profile_enable.restype = st
    L.mlb_profile_read.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]
    L.mlb_profile_read.restype = ctypes.c_int32
    L.mlb_kernel_name.argtypes = [ctypes.c_int32]
    L.mlb_kernel_name.restype = ctypes.c_char_p
    L.mlb_conservation_noalloc.argtypes = [vp, dp, ctypes.c_int32, ctypes.c_int64, vp, vp]
    L.mlb_conservation_noalloc.restype = st
    L.mlb_step_monitored.argtypes = [vp, dp]
    L.mlb_step_monitored.restype = st
    L.mlb_copy_bandwidth.argtypes = [ctypes.c_int64, ctypes.c_int32, dp]
    L.mlb_copy_bandwidth.restype = st
    L.mlb_fma_throughput.argtypes = [ctypes.c_int32, ctypes.c_int32, dp]
    L.mlb_fma_throughput.restype = st
    L.mlb_autotune.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    L.mlb_autotune.restype = st
    L.mlb_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, vp, ctypes.POINTER(vp)]
    L.mlb_batch_create.restype = st
    L.mlb_batch_step.argtypes = [vp, ctypes.c_int64]
    L.mlb_batch_step.restype = st
    L.mlb_batch_synchronize.argtypes = [vp]
    L.mlb_batch_synchronize.restype = st
    L.mlb_batch_set_grouping.argtypes = [vp, ctypes.c_int32, ctypes.c_int64]
    L.mlb_batch_set_grouping.restype = st
    L.mlb_batch_grouped_members.argtypes = [vp]
    L.mlb_batch_grouped_members.restype = ctypes.c_int32
    L.mlb_batch_last_error.argtypes = [vp]
    L.mlb_batch_last_error.restype = ctypes.c_char_p
    L.mlb_batch_destroy.argtypes = [vp]
    L.mlb_batch_destroy.restype = None
    L.mlb_get_rest_force.argtypes = [vp, dp]
    L.mlb_get_rest_force.restype = st
    L.mlb_net_param_count.argtypes = []
    L.mlb_net_param_count.restype = ctypes.c_int64
    L.mlb_net_create.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(vp)]
    L.mlb_net_create.restype = st
    L.mlb_net_set_params.argtypes = [vp, fp]
    L.mlb_net_set_params.restype = st
    L.mlb_net_get_params.argtypes = [vp, fp]
    L.mlb_net_get_params.restype = st
    L.mlb_net_set_scales.argtypes = [vp, dp, dp]
    L.mlb_net_set_scales.restype = st
    L.mlb_net_forward.argtypes = [vp, dp, dp]
    L.mlb_net_forward.restype = st
    L.mlb_net_gradient.argtypes = [vp, dp, dp, fp, dp]
    L.mlb_net_gradient.restype = st
    L.mlb_net_train.argtypes = [vp, dp, dp, ctypes.c_int32, ctypes.c_double, dp]
    L.mlb_net_train.restype = st
    L.mlb_net_last_error.argtypes = [vp]
    L.mlb_net_last_error.restype = ctypes.c_char_p
    L.mlb_net_destroy.argtypes = [vp]
    L.mlb_net_destroy.restype = None
    L.mlb_attach_surrogate.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_double]
    L.mlb_attach_surrogate.restype = st
    L.mlb_surrogate_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), dp, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64)]
    L.mlb_surrogate_status.restype = st
    L.mlb_last_error.argtypes = [vp]
    L.mlb_last_error.restype = ctypes.c_char_p
    L.mlb_status_string.argtypes = [ctypes.c_int]
    L.mlb_status_string.restype = ctypes.c_char_p
    L.mlb_destroy.argtypes = [vp]
    L.mlb_destroy.restype = None
    return L


lib = _load()


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def fma_throughput(iters: int = 1 << 14, reps: int = 10) -> float:
    """Measured FP32 FMA throughput of the current device in TFLOP/s
    (mlb_fma_throughput)."""
    out = ctypes.c_double()
    rc = lib.mlb_fma_throughput(int(iters), int(reps), ctypes.byref(out))
    if rc != 0:
        raise MLBError(rc, "mlb_fma_throughput failed")
    return out.value


def copy_bandwidth(nbytes: int = 1 << 31, reps: int = 20) -> float:
    """GB/s of the library's device-to-device float4 copy over two buffers of
    nbytes (bytes read + written per second; mlb_copy_bandwidth)."""
    out = ctypes.c_double()
    rc = lib.mlb_copy_bandwidth(int(nbytes), int(reps), ctypes.byref(out))
    if rc != 0:
        raise MLBError(rc, "mlb_copy_bandwidth failed")
    return float(out.value)


def velocity_set():
    c = np.zeros((MLB_Q, 3), np.int32)
    w = np.zeros(MLB_Q)
    lib.mlb_velocity_set(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(w))
    return c, w


class _TorchAllocator:
    """dev_alloc/dev_free callbacks backed by torch's caching allocator."""

    def __init__(self, device: int, stream_ptr: int):
        import torch
        self.torch = torch
        self.device = device
        self.stream_ptr = stream_ptr

        def alloc(nbytes, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream_ptr or None))
            except Exception:          # allocation failure -> NULL -> MLB_ENOMEM
                return None

        def free(ptr, user):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc_fn = ALLOC_FN(alloc)
        self.free_fn = FREE_FN(free)


class Simulation:
    """One mlb context for a ``workloads.Lattice``.

    stream: a torch.cuda.Stream (default: torch's current stream);
    torch_alloc: take device memory from torch's caching allocator;
    split_collide: launch pass 2 and the collision separately (MLB_SPLIT_COLLIDE)
    instead of the fused kernel; the populations are bitwise the same.
    """

    def __init__(self, lat, stream=None, torch_alloc: bool = True, split_collide: bool = False):
        import torch
        self.lat = lat
        self.S = lat.nspecies
        self.N = lat.nsites
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        d = mlb_lattice_desc()
        d.nx, d.ny, d.nz = lat.shape
        d.nspecies = self.S
        d.wall_axis = lat.wall_axis
        d.flags = (MLB_DRAG_ONLY if lat.drag_only else 0) | (
            MLB_FORCE_EXPLICIT if lat.force_scheme == "explicit" else 0) | (MLB_SPLIT_COLLIDE if split_collide else 0)
        mf = getattr(lat, "meanfield", "fp32")
        if mf not in ("fp32", "bf16", "bf16_1pass"):
            raise ValueError(f"meanfield must be fp32, bf16 or bf16_1pass, not {mf!r}")
        d.flags |= (MLB_MEANFIELD_BF16 if mf != "fp32" else 0) | (MLB_MEANFIELD_BF16_1PASS if mf == "bf16_1pass" else 0)
        for k in range(3):
            d.wall_u_lo[k] = lat.wall_u_lo[k]
            d.wall_u_hi[k] = lat.wall_u_hi[k]
        d.tau, d.kT, d.kappa = lat.tau, lat.kT, lat.kappa
        d.stream = ctypes.c_void_p(stream.cuda_stream)
        self._alloc = None
        if torch_alloc:
            self._alloc = _TorchAllocator(stream.device.index if stream.device.index is not None
                                          else torch.cuda.current_device(), stream.cuda_stream)
            d.dev_alloc = self._alloc.alloc_fn
            d.dev_free = self._alloc.free_fn
        self.ctx = ctypes.c_void_p()
        st = lib.mlb_create(ctypes.byref(d), ctypes.byref(self.ctx))
        self._check(st)
        self._check(lib.mlb_set_species(self.ctx, _dp(np.ascontiguousarray(lat.sigma, np.float64)),
                                        _dp(np.ascontiguousarray(lat.mass, np.float64))))
        eps = np.ascontiguousarray(lat.eps, np.float64)
        if np.any(eps != 0):
            self._check(lib.mlb_set_interactions(self.ctx, _dp(eps),
                                                 _dp(np.ascontiguousarray(lat.lambda_c, np.float64))))
        sweeps = int(getattr(lat, "predictor_sweeps", 1))
        if sweeps != 1:
            self._check(lib.mlb_set_predictor_sweeps(self.ctx, sweeps))

    # -- plumbing
    def _check(self, st):
        if st != 0:
            msg = lib.mlb_last_error(self.ctx).decode() if self.ctx else ""
            raise MLBError(st, msg)

    def close(self):
        if getattr(self, "ctx", None):
            lib.mlb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the ABI, with numpy arrays
    def set_fields(self, n, u=None):
        n = np.ascontiguousarray(n, np.float64).reshape(self.S, self.N)
        uu = None if u is None else np.ascontiguousarray(u, np.float64).reshape(self.S, 3, self.N)
        self._check(lib.mlb_set_fields(self.ctx, _dp(n), _dp(uu)))

    def set_external_force(self, fext):
        fe = None if fext is None else np.ascontiguousarray(fext, np.float64).reshape(self.S, 3, self.N)
        self._check(lib.mlb_set_external_force(self.ctx, _dp(fe)))

    def step(self, nsteps: int):
        self._check(lib.mlb_step(self.ctx, int(nsteps)))

    def synchronize(self):
        self._check(lib.mlb_synchronize(self.ctx))

    def moments(self, out_n=None, out_u=None):
        n = np.empty((self.S, self.N)) if out_n is None else out_n
        u = np.empty((self.S, 3, self.N)) if out_u is None else out_u
        self._check(lib.mlb_get_moments(self.ctx, _dp(n), _dp(u)))
        return n, u

    def acceleration(self):
        a = np.empty((self.S, 3, self.N))
        self._check(lib.mlb_get_acceleration(self.ctx, _dp(a)))
        return a

    def step_monitored(self, sums: np.ndarray):
        """One step; the FP64 conservation sums (mass[S], mom[3]) of the state
        it starts from land in `sums` (float64, S + 3, ideally pinned) when the
        stream gets there (mlb_step_monitored): read them after synchronize()
        or a CUDA event recorded behind the call."""
        assert sums.dtype == np.float64 and sums.flags.c_contiguous and sums.size >= self.S + 3
        self._check(lib.mlb_step_monitored(self.ctx, _dp(sums)))

    def conservation(self):
        m = np.empty(self.S)
        p = np.empty(3)
        self._check(lib.mlb_conservation(self.ctx, _dp(m), _dp(p)))
        return m, p

    def populations(self):
        f = np.empty((self.S, MLB_Q, self.N), np.float32)
        nref = np.empty(self.S)
        step = ctypes.c_int64()
        self._check(lib.mlb_get_populations(self.ctx, f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                            _dp(nref), ctypes.byref(step)))
        return f, nref, step.value

    def set_populations(self, f, nref, step=0):
        f = np.ascontiguousarray(f, np.float32)
        self._check(lib.mlb_set_populations(self.ctx, f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                            _dp(np.ascontiguousarray(nref, np.float64)), int(step)))

    def rest_force(self):
        """F^hc + G + F_ext at the current state, [S][3][N] (mlb_get_rest_force)."""
        f = np.empty((self.S, 3, self.N))
        self._check(lib.mlb_get_rest_force(self.ctx, _dp(f)))
        return f

    def attach_surrogate(self, net, recheck_every: int = 50, bound: float = 0.05):
        """Take the hard-core force from `net` (a Net; None detaches it); every
        `recheck_every` steps the exact force is used and compared, and a
        relative 2-norm error above `bound` detaches the network for good."""
        self._surrogate = net
        self._check(lib.mlb_attach_surrogate(self.ctx, net.n if net is not None else None, recheck_every, bound))

    def surrogate_status(self):
        """(active, last relative error, rechecks, rejections)."""
        a = ctypes.c_int32()
        e = ctypes.c_double()
        rc = ctypes.c_int64()
        rj = ctypes.c_int64()
        self._check(lib.mlb_surrogate_status(self.ctx, ctypes.byref(a), ctypes.byref(e), ctypes.byref(rc),
                                             ctypes.byref(rj)))
        return bool(a.value), e.value, rc.value, rj.value

    def autotune(self, trials: int = 3):
        """Pick the planes per block and the fused/split pass-2 launch by timing
        (state and results unchanged); returns (zchunk, fused)."""
        z = ctypes.c_int32()
        fu = ctypes.c_int32()
        self._check(lib.mlb_autotune(self.ctx, trials, ctypes.byref(z), ctypes.byref(fu)))
        return z.value, bool(fu.value)

    def launches_per_step(self) -> int:
        return int(lib.mlb_launches_per_step(self.ctx))

    def profile(self, enable: bool = True):
        self._check(lib.mlb_profile_enable(self.ctx, 1 if enable else 0))

    def profile_read(self):
        """{kernel name: (total ms, launches)} since the last read."""
        cap = 32
        ms = np.zeros(cap)
        cnt = np.zeros(cap, np.int64)
        k = lib.mlb_profile_read(self.ctx, _dp(ms), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap)
        if k < 0:
            raise MLBError(6, "profile read failed")
        return {lib.mlb_kernel_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(min(k, cap))}


class Batch:
    """Independent Simulations stepped together through one captured CUDA
    graph (mlb_batch_*).  The members stay usable on their own; they must
    outlive the batch.  stream: a torch.cuda.Stream (default: one the batch
    creates).  lanes: members of at most max_sites sites that take the same
    kernels step by one launch per stage and lane, 0 = every member by its
    own launches (mlb_batch_set_grouping)."""

    def __init__(self, sims, stream=None, lanes: int = 1, max_sites: int = 1 << 17):
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(self.sims))(*[s.ctx.value for s in self.sims])
        self.b = ctypes.c_void_p()
        sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        st = lib.mlb_batch_create(arr, len(self.sims), sp, ctypes.byref(self.b))
        if st != 0:
            raise MLBError(st, "mlb_batch_create failed")
        if lanes != 1 or max_sites != 1 << 17:
            self._check(lib.mlb_batch_set_grouping(self.b, int(lanes), int(max_sites)))

    def grouped_members(self) -> int:
        """Members stepped by grouped launches in the current capture."""
        return int(lib.mlb_batch_grouped_members(self.b))

    def _check(self, st):
        if st != 0:
            raise MLBError(st, lib.mlb_batch_last_error(self.b).decode() if self.b else "")

    def step(self, nsteps: int):
        self._check(lib.mlb_batch_step(self.b, nsteps))

    def synchronize(self):
        self._check(lib.mlb_batch_synchronize(self.b))

    def close(self):
        if getattr(self, "b", None):
            lib.mlb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """The learned hard-core force (mlb_net_*) for lattices of shape dims:
    3D convolutions 2 -> 32 -> 32 -> 6, BF16 activations, FP32 accumulation."""

    def __init__(self, dims):
        d = (ctypes.c_int32 * 3)(*[int(v) for v in dims])
        self.dims = tuple(int(v) for v in dims)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        self.n = ctypes.c_void_p()
        st = lib.mlb_net_create(d, ctypes.byref(self.n))
        if st != 0:
            raise MLBError(st, "mlb_net_create failed")

    @staticmethod
    def param_count() -> int:
        return int(lib.mlb_net_param_count())

    def _check(self, st):
        if st != 0:
            raise MLBError(st, lib.mlb_net_last_error(self.n).decode() if self.n else "")

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.param_count()
        self._check(lib.mlb_net_set_params(self.n, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def params(self):
        p = np.empty(self.param_count(), np.float32)
        self._check(lib.mlb_net_get_params(self.n, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return p

    def set_scales(self, in_scale, out_scale):
        self._check(lib.mlb_net_set_scales(self.n, _dp(np.ascontiguousarray(in_scale, np.float64)),
                                           _dp(np.ascontiguousarray(out_scale, np.float64))))

    def forward(self, dn):
        dn = np.ascontiguousarray(dn, np.float64).reshape(2, self.N)
        f = np.empty((2, 3, self.N))
        self._check(lib.mlb_net_forward(self.n, _dp(dn), _dp(f)))
        return f

    def gradient(self, dn, force):
        dn = np.ascontiguousarray(dn, np.float64).reshape(2, self.N)
        force = np.ascontiguousarray(force, np.float64).reshape(2, 3, self.N)
        g = np.empty(self.param_count(), np.float32)
        loss = ctypes.c_double()
        self._check(lib.mlb_net_gradient(self.n, _dp(dn), _dp(force), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                         ctypes.byref(loss)))
        return loss.value, g

    def train(self, dn, force, iters: int, lr: float) -> float:
        dn = np.ascontiguousarray(dn, np.float64).reshape(2, self.N)
        force = np.ascontiguousarray(force, np.float64).reshape(2, 3, self.N)
        loss = ctypes.c_double()
        self._check(lib.mlb_net_train(self.n, _dp(dn), _dp(force), iters, lr, ctypes.byref(loss)))
        return loss.value

    def close(self):
        if getattr(self, "n", None):
            lib.mlb_net_destroy(self.n)
            self.n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
