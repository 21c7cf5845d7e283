"""ctypes binding of the C ABI in include/hydro.h.

Argument marshalling only: every step of the hot path runs in the CUDA
library.  There is no CPU fallback -- if libhydro.so is missing or fails to
load, every entry point raises.  PyTorch supplies device memory and streams.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhydro.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_UNPHYSICAL, ERR_TIMEOUT, ERR_STATE = range(7)
MEM_HOST, MEM_DEVICE = 0, 1
WENO5, WENO7, MUSTA_FORCE = 5, 7, 2
BC_OUTFLOW, BC_PERIODIC, BC_HALO = 0, 1, 2

_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "UNPHYSICAL", 5: "TIMEOUT", 6: "STATE"}


class HydroError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hydro error %s (%d): %s" % (_NAMES.get(code, "?"), code, msg))
        self.code = code


class HydroConfig(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("scheme", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 3),
        ("split", ctypes.c_int32),
        ("nq", ctypes.c_int32),
        ("limiter", ctypes.c_int32),
        ("musta_stages", ctypes.c_int32),
        ("charwise", ctypes.c_int32),
        ("dx", ctypes.c_double * 3),
        ("origin", ctypes.c_double * 3),
        ("cs2", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("dt_fixed", ctypes.c_double),
        ("weno_eps", ctypes.c_double),
        ("eos_mass", ctypes.c_double),
    ]


def make_config(n, dx, scheme=5, bc=(0, 0, 0), cs2=1.0 / 3.0, cfl=0.3, dt_fixed=0.0, eps=1e-6,
                origin=(0.0, 0.0, 0.0), split=0, nq=1, limiter=0, musta_stages=2, charwise=0, eos_mass=0.0):
    c = HydroConfig()
    for i in range(3):
        c.n[i] = int(n[i])
        c.bc[i] = int(bc[i])
        c.dx[i] = float(dx[i])
        c.origin[i] = float(origin[i])
    c.scheme = int(scheme)
    c.split = int(split)
    c.nq = int(nq)
    c.limiter = int(limiter)
    c.musta_stages = int(musta_stages)
    c.charwise = int(charwise)
    c.cs2 = float(cs2)
    c.cfl = float(cfl)
    c.dt_fixed = float(dt_fixed)
    c.weno_eps = float(eps)
    c.eos_mass = float(eos_mass)
    return c


_lib = None


def lib():
    """Load libhydro.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libhydro.so is not built (run paper_1604_03360_gb300/build.py); "
                           "there is no fallback implementation")
    L = ctypes.CDLL(LIB_PATH)
    P, vp, i32, i64, d = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "hydro_create": ([P(HydroConfig), vp, P(vp)], i32),
        "hydro_destroy": ([vp], i32),
        "hydro_set_state": ([vp, vp, i64, i32, d], i32),
        "hydro_set_primitive": ([vp, vp, i64, i32, d], i32),
        "hydro_step": ([vp, i32, d], i32),
        "hydro_get_state": ([vp, vp, i64, i32, P(d), P(i64)], i32),
        "hydro_get_primitive": ([vp, vp, i64, i32], i32),
        "hydro_sync": ([vp], i32),
        "hydro_run_many": ([vp, i32, P(vp), P(vp), i64, i32, d, d], i32),
        "hydro_get_speeds": ([vp, P(d), P(d)], i32),
        "hydro_profile_step": ([vp, i32, d, P(d)], i32),
        "hydro_last_error": ([vp], ctypes.c_char_p),
        "hydro_launch_variants": ([i32, i32, i32], i32),
        "hydro_launch_variants_cfg": ([P(HydroConfig)], i32),
        "hydro_set_launch": ([vp, i32, i32], i32),
        "hydro_get_launch": ([vp, P(i32), P(i32), P(i32), P(i32)], i32),
        "hydro_kernels_per_step": ([vp], i32),
        "hydro_autotune": ([vp, P(d)], i32),
        "hydro_state_device_ptr": ([vp], vp),
        "hydro_field_stride": ([vp], i64),
        "hydro_version": ([], ctypes.c_char_p),
        "hydro_measure_fp64_peak": ([vp, P(d)], i32),
        "hydro_eval_rcp": ([vp, vp, i64, vp], i32),
        "hydro_forward_record": ([vp, i32, i32], i32),
        "hydro_adjoint": ([vp, vp, vp, i64, i32], i32),
        "hydro_recorded_steps": ([vp, P(i32), vp, vp], i32),
        "hydro_eps2": ([vp, vp, i64, i32, P(d), vp, i64, i32], i32),
        "hydro_batch_create": ([vp, i32, vp, P(vp)], i32),
        "hydro_batch_destroy": ([vp], i32),
        "hydro_batch_set_state": ([vp, i32, vp, i64, i32, d], i32),
        "hydro_batch_set_primitive": ([vp, i32, vp, i64, i32, d], i32),
        "hydro_batch_step": ([vp, i32], i32),
        "hydro_batch_get_state": ([vp, i32, vp, i64, i32, P(d), P(i64)], i32),
        "hydro_batch_sync": ([vp], i32),
        "hydro_batch_size": ([vp], i32),
        "hydro_batch_last_error": ([vp], ctypes.c_char_p),
        "hydro_batch_profile_step": ([vp, i32, P(d)], i32),
        "hydro_batch_set_launch": ([vp, i32, i32], i32),
        "hydro_batch_get_launch": ([vp, P(i32), P(i32), P(i32), P(i32), P(i32)], i32),
        "hydro_batch_kernels_per_step": ([vp], i32),
        "hydro_batch_autotune": ([vp, P(d)], i32),
        "hydro_halo_doubles": ([vp], i64),
        "hydro_halo_pack": ([vp, i32, i32, vp, i32], i32),
        "hydro_halo_unpack": ([vp, i32, i32, vp, i32], i32),
        "hydro_halo_fill_outflow": ([vp, i32, i32], i32),
        "hydro_stage": ([vp, i32, d], i32),
        "hydro_speed_slot": ([vp, i32, i32, vp, i32], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _stream_handle(stream):
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def as_buffer(x, writable=False):
    """(pointer, field_stride, mem) of a (5, ...) float64 array or tensor."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("need a C-contiguous float64 numpy array")
        if writable and not x.flags["WRITEABLE"]:
            raise ValueError("array is read-only")
        return ctypes.c_void_p(x.ctypes.data), x[0].size, MEM_HOST
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError("need a numpy array or a torch tensor")
    if x.dtype != torch.float64 or not x.is_contiguous():
        raise ValueError("need a contiguous float64 tensor")
    return ctypes.c_void_p(x.data_ptr()), x[0].numel(), (MEM_DEVICE if x.is_cuda else MEM_HOST)


def _flat_buffer(x, n, writable=False):
    """(pointer, mem) of a contiguous float64 buffer of at least n doubles."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"] or x.size < n:
            raise ValueError("need a C-contiguous float64 array of %d doubles" % n)
        if writable and not x.flags["WRITEABLE"]:
            raise ValueError("array is read-only")
        return ctypes.c_void_p(x.ctypes.data), MEM_HOST
    import torch
    if not isinstance(x, torch.Tensor) or x.dtype != torch.float64 or not x.is_contiguous() or x.numel() < n:
        raise ValueError("need a contiguous float64 tensor of %d doubles" % n)
    return ctypes.c_void_p(x.data_ptr()), (MEM_DEVICE if x.is_cuda else MEM_HOST)


def measure_fp64_peak(stream=None):
    """FP64 FMA/s of the current device (measured by a probe kernel)."""
    L = lib()
    r = ctypes.c_double()
    rc = L.hydro_measure_fp64_peak(_stream_handle(stream), ctypes.byref(r))
    if rc:
        raise HydroError(rc, "FP64 peak probe failed")
    return r.value


def eval_rcp(x, out=None, stream=None):
    """The kernels' reciprocal (MUFU seed + one cubic Newton correction) of
    every element of the CUDA float64 tensor x (a self-check of the device
    arithmetic; the result is ordered on `stream`)."""
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
        raise ValueError("need a contiguous float64 CUDA tensor")
    y = torch.empty_like(x) if out is None else out
    rc = lib().hydro_eval_rcp(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.numel(),
                              _stream_handle(stream))
    if rc:
        raise HydroError(rc, "hydro_eval_rcp failed")
    return y


class Hydro:
    """One grid of the FP64 WENO5/WENO7 + SSP-RK3 solver (hydro_t)."""

    def __init__(self, n, dx, scheme=5, bc=(0, 0, 0), cs2=1.0 / 3.0, cfl=0.3, dt_fixed=0.0, eps=1e-6,
                 origin=(0.0, 0.0, 0.0), split=0, nq=1, limiter=0, musta_stages=2, charwise=0, eos_mass=0.0,
                 stream=None):
        self._L = lib()
        self.cfg = make_config(n, dx, scheme, bc, cs2, cfl, dt_fixed, eps, origin, split, nq, limiter, musta_stages,
                               charwise, eos_mass)
        self.n = tuple(int(k) for k in n)
        self.shape = (4 + max(1, int(nq)), self.n[2], self.n[1], self.n[0])
        h = ctypes.c_void_p()
        rc = self._L.hydro_create(ctypes.byref(self.cfg), _stream_handle(stream), ctypes.byref(h))
        if rc:
            raise HydroError(rc, self._L.hydro_last_error(None).decode())
        self._h = h
        self.t = 0.0
        self.steps = 0

    @classmethod
    def from_grid(cls, g, stream=None):
        """Create from a workloads.Grid description."""
        return cls(g.n, g.dx, scheme=g.scheme, bc=g.bc, cs2=g.cs2, cfl=g.cfl, eps=g.eps, origin=g.origin,
                   dt_fixed=getattr(g, "dt_fixed", 0.0), split=getattr(g, "split", 0), nq=getattr(g, "nq", 1),
                   limiter=getattr(g, "limiter", 0), musta_stages=getattr(g, "musta_stages", 2),
                   charwise=getattr(g, "charwise", 0), eos_mass=getattr(g, "mass", 0.0), stream=stream)

    def _check(self, rc):
        if rc:
            raise HydroError(rc, self._L.hydro_last_error(self._h).decode())

    def set_state(self, u, t=0.0):
        p, fs, mem = as_buffer(u)
        self._check(self._L.hydro_set_state(self._h, p, fs, mem, float(t)))
        self.t, self.steps = float(t), 0

    def set_primitive(self, w, t=0.0):
        p, fs, mem = as_buffer(w)
        self._check(self._L.hydro_set_primitive(self._h, p, fs, mem, float(t)))
        self.t, self.steps = float(t), 0

    def step(self, nsteps=1, t_end=-1.0):
        self._check(self._L.hydro_step(self._h, int(nsteps), float(t_end)))

    def profile_step(self, nsteps=1, t_end=-1.0):
        """Per-kernel device ms (step-begin, stage 1..3, step-end) summed over nsteps."""
        ms = (ctypes.c_double * 5)()
        self._check(self._L.hydro_profile_step(self._h, int(nsteps), float(t_end), ms))
        return np.array(ms[:])

    def autotune(self):
        """Time the compiled tile shapes / z-chunks on this grid; keep the fastest."""
        ms = ctypes.c_double()
        self._check(self._L.hydro_autotune(self._h, ctypes.byref(ms)))
        return ms.value

    def set_launch(self, variant, zc=0):
        self._check(self._L.hydro_set_launch(self._h, int(variant), int(zc)))

    def launch(self):
        """(variant, tile_x, tile_y, z_chunk) of the stage kernel."""
        v = [ctypes.c_int32() for _ in range(4)]
        self._check(self._L.hydro_get_launch(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def kernels_per_step(self):
        """Kernels one step launches with the current launch configuration."""
        return int(self._L.hydro_kernels_per_step(self._h))

    def forward_record(self, nsteps, ckpt_every=10):
        """Advance nsteps steps, recording speeds/dt and checkpoints for adjoint()."""
        self._check(self._L.hydro_forward_record(self._h, int(nsteps), int(ckpt_every)))

    def adjoint(self, lam, out=None):
        """(d u_N / d u_0)^T lam for the recorded run (frozen speeds and dt)."""
        if out is None:
            out = np.empty(self.shape) if isinstance(lam, np.ndarray) else lam.new_empty(lam.shape)
        pl, fs, mem = as_buffer(lam)
        po, fo, memo = as_buffer(out, writable=True)
        if fs != fo or mem != memo:
            raise ValueError("lam and out must have the same layout and memory kind")
        self._check(self._L.hydro_adjoint(self._h, pl, po, fs, mem))
        return out

    def recorded_steps(self):
        n = ctypes.c_int32()
        self._check(self._L.hydro_recorded_steps(self._h, ctypes.byref(n), None, None))
        al = np.empty((max(n.value, 1), 3, 3))
        dt = np.empty(max(n.value, 1))
        self._check(self._L.hydro_recorded_steps(self._h, ctypes.byref(n), ctypes.c_void_p(al.ctypes.data),
                                                 ctypes.c_void_p(dt.ctypes.data)))
        return al[:n.value], dt[:n.value]

    def eps2(self, u=None, grad=None):
        """eps_2 of u (default: the current state); fills grad (same layout) if given."""
        e = ctypes.c_double()
        if u is not None:
            pu, fu, mu = as_buffer(u)
        else:
            pu, fu, mu = None, 0, 0
        if grad is not None:
            pg, fg, mg = as_buffer(grad, writable=True)
        else:
            pg, fg, mg = None, 0, 0
        self._check(self._L.hydro_eps2(self._h, pu, fu, mu, ctypes.byref(e), pg, fg, mg))
        return e.value

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        p, fs, mem = as_buffer(out, writable=True)
        t = ctypes.c_double()
        k = ctypes.c_int64()
        self._check(self._L.hydro_get_state(self._h, p, fs, mem, ctypes.byref(t), ctypes.byref(k)))
        self.t, self.steps = t.value, k.value
        return out

    def get_primitive(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        p, fs, mem = as_buffer(out, writable=True)
        self._check(self._L.hydro_get_primitive(self._h, p, fs, mem))
        return out

    def sync(self):
        self._check(self._L.hydro_sync(self._h))

    def run_many(self, inputs, outputs, nsteps=1, t0=0.0, t_end=-1.0):
        """Event-by-event stream: load each host state of `inputs`, advance
        nsteps RK3 steps from t0 and write the result into the matching host
        buffer of `outputs` (page-locked buffers overlap the copies with the
        steps).  All buffers share one field stride."""
        if len(inputs) != len(outputs):
            raise ValueError("one output buffer per input")
        n = len(inputs)
        pin, pout, fs = (ctypes.c_void_p * max(n, 1))(), (ctypes.c_void_p * max(n, 1))(), None
        for i, (a, b) in enumerate(zip(inputs, outputs)):
            pa, fa, ma = as_buffer(a)
            pb, fb, mb = as_buffer(b, writable=True)
            if ma != MEM_HOST or mb != MEM_HOST:
                raise ValueError("run_many streams host buffers")
            if fa != fb or (fs is not None and fa != fs):
                raise ValueError("all buffers need the same field stride")
            fs = fa
            pin[i], pout[i] = pa, pb
        self._check(self._L.hydro_run_many(self._h, n, pin, pout, int(fs or 0), int(nsteps), float(t0),
                                           float(t_end)))

    # -- z-slab (bc[2] = BC_HALO) handles: one RK stage at a time ---------

    def halo_doubles(self):
        """Doubles in one side's ghost block (0 for a whole grid)."""
        return int(self._L.hydro_halo_doubles(self._h))

    def halo_pack(self, level, side, buf):
        """Interior planes next to `side` of RK level `level` -> buf (1-D float64)."""
        p, mem = _flat_buffer(buf, self.halo_doubles(), writable=True)
        self._check(self._L.hydro_halo_pack(self._h, int(level), int(side), p, mem))
        return buf

    def halo_unpack(self, level, side, buf):
        """buf (a neighbour's pack) -> ghost planes on `side` of level `level`."""
        p, mem = _flat_buffer(buf, self.halo_doubles())
        self._check(self._L.hydro_halo_unpack(self._h, int(level), int(side), p, mem))

    def halo_fill_outflow(self, level, side):
        self._check(self._L.hydro_halo_fill_outflow(self._h, int(level), int(side)))

    def stage(self, which, t_end=-1.0):
        """0 step begin, 1..3 RK stage, 4 step commit."""
        self._check(self._L.hydro_stage(self._h, int(which), float(t_end)))

    def speed_slot(self, slot, buf=None, write=False):
        """Read (or, write=True, overwrite) speed slot 0..3 through a 3-double buffer."""
        if buf is None:
            buf = np.zeros(3)
        p, mem = _flat_buffer(buf, 3, writable=not write)
        self._check(self._L.hydro_speed_slot(self._h, int(slot), 1 if write else 0, p, mem))
        return buf

    def speeds(self):
        a = (ctypes.c_double * 3)()
        dt = ctypes.c_double()
        self._check(self._L.hydro_get_speeds(self._h, a, ctypes.byref(dt)))
        return np.array(a[:]), dt.value

    def close(self):
        if getattr(self, "_h", None):
            self._L.hydro_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class HydroBatch:
    """An event-by-event ensemble of independent grids (hydro_batch_t): one
    persistent launch per RK3 stage walks a work-list of all events' tiles."""

    def __init__(self, grids, stream=None):
        """grids: sequence of workloads.Grid (or objects with n, dx, scheme, bc,
        cs2, cfl, eps, origin)."""
        self._L = lib()
        self.grids = list(grids)
        arr = (HydroConfig * len(self.grids))()
        for i, g in enumerate(self.grids):
            arr[i] = make_config(g.n, g.dx, g.scheme, g.bc, g.cs2, g.cfl, getattr(g, "dt_fixed", 0.0), g.eps,
                                 g.origin, getattr(g, "split", 0), getattr(g, "nq", 1), getattr(g, "limiter", 0),
                                 getattr(g, "musta_stages", 2), getattr(g, "charwise", 0), getattr(g, "mass", 0.0))
        h = ctypes.c_void_p()
        rc = self._L.hydro_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(self.grids), _stream_handle(stream),
                                        ctypes.byref(h))
        if rc:
            raise HydroError(rc, self._L.hydro_batch_last_error(None).decode())
        self._h = h
        self.shapes = [(5, g.n[2], g.n[1], g.n[0]) for g in self.grids]

    def __len__(self):
        return len(self.grids)

    def _check(self, rc):
        if rc:
            raise HydroError(rc, self._L.hydro_batch_last_error(self._h).decode())

    def set_state(self, e, u, t=0.0):
        p, fs, mem = as_buffer(u)
        self._check(self._L.hydro_batch_set_state(self._h, int(e), p, fs, mem, float(t)))

    def set_primitive(self, e, w, t=0.0):
        p, fs, mem = as_buffer(w)
        self._check(self._L.hydro_batch_set_primitive(self._h, int(e), p, fs, mem, float(t)))

    def step(self, nsteps=1):
        self._check(self._L.hydro_batch_step(self._h, int(nsteps)))

    def get_state(self, e, out=None):
        if out is None:
            out = np.empty(self.shapes[e])
        p, fs, mem = as_buffer(out, writable=True)
        t = ctypes.c_double()
        k = ctypes.c_int64()
        self._check(self._L.hydro_batch_get_state(self._h, int(e), p, fs, mem, ctypes.byref(t), ctypes.byref(k)))
        return out, t.value, k.value

    def sync(self):
        self._check(self._L.hydro_batch_sync(self._h))

    def profile_step(self, nsteps=1):
        ms = (ctypes.c_double * 5)()
        self._check(self._L.hydro_batch_profile_step(self._h, int(nsteps), ms))
        return np.array(ms[:])

    def autotune(self):
        ms = ctypes.c_double()
        self._check(self._L.hydro_batch_autotune(self._h, ctypes.byref(ms)))
        return ms.value

    def set_launch(self, variant, zc=0):
        self._check(self._L.hydro_batch_set_launch(self._h, int(variant), int(zc)))

    def launch(self):
        """(variant, tile_x, tile_y, z_chunk, work items)."""
        v = [ctypes.c_int32() for _ in range(5)]
        self._check(self._L.hydro_batch_get_launch(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def kernels_per_step(self):
        """Kernels one step launches (the whole batch)."""
        return int(self._L.hydro_batch_kernels_per_step(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._L.hydro_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
