"""Thin ctypes binding of the C ABI in include/mm.h (argument marshalling only).

Every computation runs in the CUDA library ``_build/libmm.so``; if it is
missing this module raises at import time -- there is no CPU fallback.
Module-level functions carry the ABI's names; ``Context`` wraps a handle and
``Context.from_problem`` configures one from a ``workloads.Problem``.
Arrays cross the boundary as float32 SoA (3, nz, ny, nx) and uint8 maps
(nz, ny, nx); device variants take torch CUDA tensors (memory only).
"""
import ctypes as C
import os

import numpy as np

from .build import LIB

if not os.path.exists(LIB):
    raise ImportError(f"CUDA library not built ({LIB}); run paper_1406_7635_gb300.build.build()")

_lib = C.CDLL(LIB)

MM_OK = 0
MM_RK45, MM_RK23 = 0, 1
ERRORS = {-1: "MM_ERR_ARG", -2: "MM_ERR_CUDA", -3: "MM_ERR_OOM", -4: "MM_ERR_NONFINITE",
          -5: "MM_ERR_DT_UNDERFLOW", -6: "MM_ERR_TIMEOUT", -7: "MM_ERR_STATE"}


class MMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class mm_material(C.Structure):
    _fields_ = [("msat", C.c_double), ("aex", C.c_double), ("alpha", C.c_double), ("gamma_ll", C.c_double),
                ("ku1", C.c_double), ("ku2", C.c_double), ("anis_u", C.c_double * 3), ("dind", C.c_double),
                ("jcur", C.c_double * 3), ("xi", C.c_double), ("pol", C.c_double), ("lambda_sl", C.c_double),
                ("eps_prime", C.c_double), ("mp", C.c_double * 3), ("tfree", C.c_double)]


class mm_energies(C.Structure):
    _fields_ = [("total", C.c_double), ("demag", C.c_double), ("exch", C.c_double), ("anis", C.c_double),
                ("zeeman", C.c_double), ("m_avg", C.c_double * 3), ("dmi", C.c_double)]


class mm_stats(C.Structure):
    _fields_ = [("accepted", C.c_longlong), ("rejected", C.c_longlong), ("evals", C.c_longlong),
                ("last_err", C.c_double), ("t", C.c_double), ("dt", C.c_double), ("launches", C.c_longlong)]


class mm_instance_spec(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dz", C.c_double), ("msat", C.c_double), ("aex", C.c_double), ("alpha", C.c_double),
                ("gamma_ll", C.c_double), ("bext", C.c_double * 3)]


class mm_fno_cfg(C.Structure):
    _fields_ = [("width", C.c_int), ("layers", C.c_int), ("modes_x", C.c_int), ("modes_y", C.c_int),
                ("max_batch", C.c_int), ("seed", C.c_ulonglong)]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_SIGS = {
    "mm_last_error": (C.c_char_p, []),
    "mm_create": (_I, [C.POINTER(_P), _I, _I, _I, _D, _D, _D, _I, _P]),
    "mm_destroy": (_I, [_P]),
    "mm_set_geometry": (_I, [_P, _P]),
    "mm_set_regions": (_I, [_P, _P]),
    "mm_set_region_material": (_I, [_P, _I, C.POINTER(mm_material)]),
    "mm_set_exchange_scale": (_I, [_P, _I, _I, _D]),
    "mm_set_bext": (_I, [_P, _I, _P, _P]),
    "mm_set_bext_timefn": (_I, [_P, _D, _D]),
    "mm_enable_terms": (_I, [_P, _I, _I, _I, _I, _I]),
    "mm_set_m": (_I, [_P, _P]),
    "mm_get_m": (_I, [_P, _P]),
    "mm_set_m_device": (_I, [_P, _P]),
    "mm_get_m_device": (_I, [_P, _P]),
    "mm_set_solver": (_I, [_P, _D, _D, _D, _D, _D]),
    "mm_set_fixed_dt_sequence": (_I, [_P, _P, _I]),
    "mm_set_wait_limit": (_I, [_P, C.c_longlong]),
    "mm_get_wait_limit": (_I, [_P, C.POINTER(C.c_longlong)]),
    "mm_step": (_I, [_P, _I]),
    "mm_run": (_I, [_P, _D]),
    "mm_get_time": (_I, [_P, C.POINTER(_D), C.POINTER(_D)]),
    "mm_set_time": (_I, [_P, _D, _D]),
    "mm_get_beff": (_I, [_P, _P]),
    "mm_get_bdemag": (_I, [_P, _P]),
    "mm_get_torque": (_I, [_P, _P]),
    "mm_get_energies": (_I, [_P, C.POINTER(mm_energies)]),
    "mm_get_stats": (_I, [_P, C.POINTER(mm_stats)]),
    "mm_get_max_torque": (_I, [_P, C.POINTER(_D)]),
    "mm_set_pbc": (_I, [_P, _I, _I, _I]),
    "mm_enable_stt": (_I, [_P, _I, _I]),
    "mm_set_integrator": (_I, [_P, _I]),
    "mm_get_integrator": (_I, [_P, C.POINTER(_I)]),
    "mm_relax": (_I, [_P, C.c_longlong, C.POINTER(C.c_longlong)]),
    "mm_get_dt_history": (_I, [_P, _P, _I, C.POINTER(_I)]),
    "mm_state_bytes": (C.c_size_t, [_P]),
    "mm_get_state": (_I, [_P, _P, C.c_size_t]),
    "mm_set_state": (_I, [_P, _P, C.c_size_t]),
    "mm_demag_tensor": (_I, [_I, _D, _D, _D, _I, _P, _P]),
    "mm_demag_apply": (_I, [_P, _P, _P]),
    "mm_demag_field_noalloc": (_I, [_I, _I, _I, _D, _D, _D, _P, _P, _P]),
    "mm_sync": (_I, [_P]),
    "mm_profile_attempts": (_I, [_P, _I, _I, _P, _P, C.POINTER(_I)]),
    "mm_set_yz_kernels": (_I, [_P, _I, C.POINTER(_I)]),
    "mm_fp32_peak": (_I, [_I, _I, C.POINTER(_D), C.POINTER(_I), C.POINTER(_I)]),
    "mm_batch_create": (_I, [C.POINTER(_P), _I, C.POINTER(mm_instance_spec), _I, _P]),
    "mm_batch_destroy": (_I, [_P]),
    "mm_batch_set_m": (_I, [_P, _I, _P]),
    "mm_batch_get_m": (_I, [_P, _I, _P]),
    "mm_batch_set_solver": (_I, [_P, _D, _D, _D, _D, _D]),
    "mm_batch_run": (_I, [_P, _D]),
    "mm_batch_get_stats": (_I, [_P, _I, C.POINTER(mm_stats)]),
    "mm_batch_get_dt_history": (_I, [_P, _I, _P, _I, C.POINTER(_I)]),
    "mm_batch_num_classes": (_I, [_P]),
    "mm_batch_class_info": (_I, [_P, _I, _P, C.POINTER(_D)]),
    "mm_batch_set_tiles": (_I, [_P, _I, _I, _I, _I]),
    "mm_fno_create": (_I, [C.POINTER(_P), _I, _I, C.POINTER(mm_fno_cfg), _I, _P]),
    "mm_fno_destroy": (_I, [_P]),
    "mm_fno_param_count": (C.c_longlong, [_P]),
    "mm_fno_get_params": (_I, [_P, _P, C.c_longlong]),
    "mm_fno_set_params": (_I, [_P, _P, C.c_longlong]),
    "mm_fno_forward": (_I, [_P, _P, _P, _I]),
    "mm_fno_grad": (_I, [_P, _P, _P, _I, _P, C.POINTER(_D)]),
    "mm_fno_train_step": (_I, [_P, _P, _P, _I, _D, C.POINTER(_D)]),
    "mm_surrogate_train": (_I, [_P, _P, _D, _I, _I, _I, _D, _I, _I, _D, C.c_ulonglong, C.POINTER(_D)]),
    "mm_set_demag_surrogate": (_I, [_P, _P, _D, _I, _D]),
    "mm_get_surrogate_stats": (_I, [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                    C.POINTER(C.c_longlong), C.POINTER(_D), C.POINTER(_I)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = sorted(_SIGS)


def _check(rc):
    if rc != MM_OK:
        raise MMError(rc, mm_last_error().decode())
    return rc


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def demag_tensor(offsets, dx, dy, dz, device=0):
    """N_ij (float64, [n, 6]) for integer offsets [n, 3] computed on the GPU."""
    off = np.ascontiguousarray(offsets, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((off.shape[0], 6), dtype=np.float64)
    _check(mm_demag_tensor(device, dx, dy, dz, off.shape[0], _ptr(off), _ptr(out)))
    return out


def demag_field_noalloc(M_dev, B_dev, nx, ny, nz, dx, dy, dz, stream=None):
    """B (device tensor) of M (device tensor, A/m) using only the library's
    static scratch: no device allocation (see mm_demag_field_noalloc)."""
    _check(mm_demag_field_noalloc(nx, ny, nz, dx, dy, dz, C.c_void_p(M_dev.data_ptr()),
                                  C.c_void_p(B_dev.data_ptr()), stream))


def fp32_peak(device=0, reps=5):
    """Measured FP32 FMA throughput (TFLOP/s), SM count and maximum SM clock
    (MHz) of a device (mm_fp32_peak)."""
    tf, sms, mhz = C.c_double(), C.c_int(), C.c_int()
    _check(mm_fp32_peak(device, reps, C.byref(tf), C.byref(sms), C.byref(mhz)))
    return tf.value, sms.value, mhz.value


KERNEL_KINDS = {0: "prep", 1: "yz", 2: "row", 3: "yf", 4: "zk", 5: "yi", 6: "part"}


class Context:
    """A grid, its materials and its integrator state on one GPU."""

    def __init__(self, nx, ny, nz, dx, dy, dz, device=0, stream=None):
        h = C.c_void_p()
        _check(mm_create(C.byref(h), nx, ny, nz, dx, dy, dz, device, stream))
        self.h = h
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz

    def close(self):
        if self.h:
            mm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- set-up ---
    def set_geometry(self, mask):
        a = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(self.shape)
        _check(mm_set_geometry(self.h, None if a is None else _ptr(a)))

    def set_regions(self, region):
        a = None if region is None else np.ascontiguousarray(region, dtype=np.uint8).reshape(self.shape)
        _check(mm_set_regions(self.h, None if a is None else _ptr(a)))

    def set_material(self, region, msat, aex, alpha, gamma_ll=1.7595e11, ku1=0.0, ku2=0.0, anis_u=(1.0, 0.0, 0.0),
                     dind=0.0, jcur=(0.0, 0.0, 0.0), xi=0.0, pol=0.0, lambda_sl=1.0, eps_prime=0.0,
                     mp=(0.0, 0.0, 1.0), tfree=0.0):
        m = mm_material(msat, aex, alpha, gamma_ll, ku1, ku2, (C.c_double * 3)(*anis_u), dind,
                        (C.c_double * 3)(*jcur), xi, pol, lambda_sl, eps_prime, (C.c_double * 3)(*mp), tfree)
        _check(mm_set_region_material(self.h, region, C.byref(m)))

    def set_exchange_scale(self, r1, r2, s):
        _check(mm_set_exchange_scale(self.h, r1, r2, s))

    def set_bext(self, region, b0, b1=None):
        a0 = np.ascontiguousarray(b0, dtype=np.float64)
        a1 = None if b1 is None else np.ascontiguousarray(b1, dtype=np.float64)
        _check(mm_set_bext(self.h, region, _ptr(a0), None if a1 is None else _ptr(a1)))

    def set_bext_timefn(self, freq, phase=0.0):
        _check(mm_set_bext_timefn(self.h, freq, phase))

    def enable_terms(self, demag=True, exch=True, anis=True, zeeman=True, precession=True):
        _check(mm_enable_terms(self.h, int(demag), int(exch), int(anis), int(zeeman), int(precession)))

    def set_solver(self, max_err=1e-5, headroom=0.8, dt0=1e-14, dt_min=1e-20, dt_max=1e-10):
        _check(mm_set_solver(self.h, max_err, headroom, dt0, dt_min, dt_max))

    def set_fixed_dt_sequence(self, dts):
        a = np.ascontiguousarray(dts, dtype=np.float64)
        _check(mm_set_fixed_dt_sequence(self.h, _ptr(a) if a.size else None, a.size))

    def set_wait_limit(self, cycles):
        _check(mm_set_wait_limit(self.h, int(cycles)))

    def get_wait_limit(self):
        v = C.c_longlong()
        _check(mm_get_wait_limit(self.h, C.byref(v)))
        return v.value

    # --- state ---
    def set_m(self, m):
        a = np.ascontiguousarray(m, dtype=np.float32).reshape((3,) + self.shape)
        _check(mm_set_m(self.h, _ptr(a)))

    def get_m(self, out=None):
        """m as float32 [3][nz][ny][nx]; into `out` (a C-contiguous float32
        array of that shape, e.g. in pinned memory) when given."""
        if out is None:
            out = np.zeros((3,) + self.shape, dtype=np.float32)
        elif out.dtype != np.float32 or out.shape != (3,) + self.shape or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a C-contiguous float32 array of shape (3, nz, ny, nx)")
        _check(mm_get_m(self.h, _ptr(out)))
        return out

    def set_m_device(self, t):
        assert t.is_cuda and t.dtype.itemsize == 4 and t.is_contiguous() and t.numel() == 3 * self.n
        _check(mm_set_m_device(self.h, C.c_void_p(t.data_ptr())))

    def get_m_device(self, t):
        assert t.is_cuda and t.dtype.itemsize == 4 and t.is_contiguous() and t.numel() == 3 * self.n
        _check(mm_get_m_device(self.h, C.c_void_p(t.data_ptr())))

    def step(self, n):
        _check(mm_step(self.h, int(n)))

    def run(self, t_end):
        _check(mm_run(self.h, float(t_end)))

    def get_time(self):
        t, dt = C.c_double(), C.c_double()
        _check(mm_get_time(self.h, C.byref(t), C.byref(dt)))
        return t.value, dt.value

    def set_time(self, t, dt):
        _check(mm_set_time(self.h, t, dt))

    def _vec(self, fn):
        out = np.zeros((3,) + self.shape, dtype=np.float32)
        _check(fn(self.h, _ptr(out)))
        return out

    def get_beff(self):
        return self._vec(mm_get_beff)

    def get_bdemag(self):
        return self._vec(mm_get_bdemag)

    def get_torque(self):
        return self._vec(mm_get_torque)

    def get_energies(self):
        e = mm_energies()
        _check(mm_get_energies(self.h, C.byref(e)))
        return {"total": e.total, "demag": e.demag, "exch": e.exch, "anis": e.anis, "zeeman": e.zeeman,
                "dmi": e.dmi, "m_avg": list(e.m_avg)}

    def enable_stt(self, zhang_li, slonczewski):
        _check(mm_enable_stt(self.h, int(bool(zhang_li)), int(bool(slonczewski))))

    def set_pbc(self, px, py, pz):
        _check(mm_set_pbc(self.h, int(px), int(py), int(pz)))

    def get_max_torque(self):
        v = C.c_double()
        _check(mm_get_max_torque(self.h, C.byref(v)))
        return v.value

    def set_integrator(self, method):
        _check(mm_set_integrator(self.h, {"rk45": MM_RK45, "rk23": MM_RK23}.get(method, method)))

    def get_integrator(self):
        v = C.c_int()
        _check(mm_get_integrator(self.h, C.byref(v)))
        return v.value

    def relax(self, max_steps=1_000_000):
        """The paper's relax(); returns the accepted steps it took."""
        n = C.c_longlong()
        _check(mm_relax(self.h, int(max_steps), C.byref(n)))
        return n.value

    def get_stats(self):
        s = mm_stats()
        _check(mm_get_stats(self.h, C.byref(s)))
        return {"accepted": s.accepted, "rejected": s.rejected, "evals": s.evals, "last_err": s.last_err,
                "t": s.t, "dt": s.dt, "launches": s.launches}

    def get_dt_history(self, max_n=1 << 20):
        out = np.zeros(max_n, dtype=np.float64)
        n = C.c_int()
        _check(mm_get_dt_history(self.h, _ptr(out), max_n, C.byref(n)))
        return out[:n.value].copy()

    def get_state(self):
        nb = mm_state_bytes(self.h)
        buf = np.zeros(nb, dtype=np.uint8)
        _check(mm_get_state(self.h, _ptr(buf), nb))
        return buf

    def set_state(self, buf):
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(mm_set_state(self.h, _ptr(b), b.size))

    def demag_apply(self, m_dev, b_dev):
        """B_demag of the device tensor m_dev into b_dev (torch CUDA, float32)."""
        _check(mm_demag_apply(self.h, C.c_void_p(m_dev.data_ptr()), C.c_void_p(b_dev.data_ptr())))

    def sync(self):
        _check(mm_sync(self.h))

    def set_yz_kernels(self, which):
        """(y, z) kernels of the convolution: 0 default, 1 cluster kernel, 2
        three kernels; returns the kernels in use (mm_set_yz_kernels)."""
        a = C.c_int()
        _check(mm_set_yz_kernels(self.h, int(which), C.byref(a)))
        return a.value

    def profile_attempts(self, attempts):
        """Per launch position of one RK45 attempt: (kind, mean microseconds)
        over `attempts` attempts launched one kernel at a time with events
        between them (mm_profile_attempts); the state advances as by
        step(attempts)."""
        kinds = np.zeros(64, dtype=np.int32)
        us = np.zeros(64, dtype=np.float64)
        n = C.c_int()
        _check(mm_profile_attempts(self.h, int(attempts), 64, _ptr(kinds), _ptr(us), C.byref(n)))
        return [(KERNEL_KINDS[int(k)], float(u)) for k, u in zip(kinds[:n.value], us[:n.value])]

    def set_demag_surrogate(self, net, ms_ref, check_every=10, fallback_rel_err=1e-3):
        _check(mm_set_demag_surrogate(self.h, None if net is None else net.h, ms_ref, check_every,
                                      fallback_rel_err))

    def surrogate_stats(self):
        a, b, c_ = C.c_longlong(), C.c_longlong(), C.c_longlong()
        e, act = C.c_double(), C.c_int()
        _check(mm_get_surrogate_stats(self.h, C.byref(a), C.byref(b), C.byref(c_), C.byref(e), C.byref(act)))
        return {"steps": a.value, "checks": b.value, "fallbacks": c_.value, "last_rel_err": e.value,
                "active": bool(act.value)}

    def train_surrogate(self, net, ms_ref, n_pairs, traj_len, steps_between, field_max, epochs, batch, lr, seed=0):
        loss = C.c_double()
        _check(mm_surrogate_train(self.h, net.h, ms_ref, n_pairs, traj_len, steps_between, field_max, epochs, batch,
                                  lr, seed, C.byref(loss)))
        return loss.value

    # --- configuration from a Problem description ---
    @classmethod
    def from_problem(cls, p, device=0, stream=None, regions_used=None):
        ctx = cls(p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, device, stream)
        if any(getattr(p, "pbc", (0, 0, 0))):
            ctx.set_pbc(*p.pbc)
        ctx.set_geometry(p.mask)
        ctx.set_regions(p.region)
        used = np.unique(p.region) if regions_used is None else regions_used
        for r in used:
            r = int(r)
            ctx.set_material(r, p.msat[r], p.aex[r], p.alpha[r], p.gamma[r], p.ku1[r], p.ku2[r], p.anis_u[r],
                             p.dind[r], p.jcur[r], p.xi[r], p.pol[r], p.lam[r], p.epsp[r], p.mp[r], p.tfree[r])
            ctx.set_bext(r, p.b0[r], p.b1[r])
        for i, r1 in enumerate(used):
            for r2 in used[i + 1:]:
                s = p.exch_scale[int(r1), int(r2)]
                if s != 1.0:
                    ctx.set_exchange_scale(int(r1), int(r2), s)
        ctx.set_bext_timefn(p.freq, p.phase)
        ctx.enable_terms(p.demag, p.exch, p.anis, p.zeeman, p.precession)
        if p.zhang_li or p.slonczewski:
            ctx.enable_stt(p.zhang_li, p.slonczewski)
        ctx.set_solver(p.max_err, p.headroom, p.dt0, p.dt_min, p.dt_max)
        ctx.set_m(p.m0)
        return ctx


class Batch:
    """Independent simulations of uneven grids advanced together (mm_batch_*).

    specs: sequence of dicts with nx, ny, nz, dx, dy, dz, msat, aex, alpha,
    gamma_ll (optional), bext (3-vector)."""

    def __init__(self, specs, device=0, stream=None):
        arr = (mm_instance_spec * len(specs))()
        self.shapes = []
        for a, s in zip(arr, specs):
            a.nx, a.ny, a.nz = s["nx"], s["ny"], s["nz"]
            a.dx, a.dy, a.dz = s["dx"], s["dy"], s["dz"]
            a.msat, a.aex, a.alpha = s["msat"], s["aex"], s["alpha"]
            a.gamma_ll = s.get("gamma_ll", 1.7595e11)
            a.bext = (C.c_double * 3)(*s["bext"])
            self.shapes.append((s["nz"], s["ny"], s["nx"]))
        h = C.c_void_p()
        _check(mm_batch_create(C.byref(h), len(specs), arr, device, stream))
        self.h = h
        self.n = len(specs)

    def close(self):
        if self.h:
            mm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_m(self, i, m):
        a = np.ascontiguousarray(m, dtype=np.float32).reshape((3,) + self.shapes[i])
        _check(mm_batch_set_m(self.h, i, _ptr(a)))

    def get_m(self, i):
        out = np.zeros((3,) + self.shapes[i], dtype=np.float32)
        _check(mm_batch_get_m(self.h, i, _ptr(out)))
        return out

    def set_solver(self, max_err=1e-5, headroom=0.8, dt0=1e-14, dt_min=1e-20, dt_max=1e-10):
        _check(mm_batch_set_solver(self.h, max_err, headroom, dt0, dt_min, dt_max))

    def run(self, t_end):
        _check(mm_batch_run(self.h, float(t_end)))

    def get_stats(self, i):
        s = mm_stats()
        rc = mm_batch_get_stats(self.h, i, C.byref(s))
        return {"accepted": s.accepted, "rejected": s.rejected, "evals": s.evals, "last_err": s.last_err,
                "t": s.t, "dt": s.dt, "status": rc}

    def get_dt_history(self, i, max_n=4096):
        out = np.zeros(max_n, dtype=np.float64)
        n = C.c_int()
        _check(mm_batch_get_dt_history(self.h, i, _ptr(out), max_n, C.byref(n)))
        return out[:n.value].copy()

    def class_info(self, c):
        """Autotuned FFT tiles of shape class c: grid, instances, residue
        split, x rows per block and the chosen convolution time (us)."""
        info = np.zeros(7, dtype=np.int32)
        us = C.c_double()
        _check(mm_batch_class_info(self.h, int(c), _ptr(info), C.byref(us)))
        return {"grid": [int(info[0]), int(info[1]), int(info[2])], "instances": int(info[3]),
                "cly": int(info[4]), "clz": int(info[5]), "xrows": int(info[6]), "conv_us": us.value}

    def num_classes(self):
        return mm_batch_num_classes(self.h)

    def set_tiles(self, c, cly, clz, xrows):
        """Pin the FFT tiles of shape class c (one of the offered splits and
        x-row block sizes)."""
        _check(mm_batch_set_tiles(self.h, int(c), int(cly), int(clz), int(xrows)))


class FNO:
    """Fourier-neural-operator demag surrogate on the GPU (mm_fno_*)."""

    def __init__(self, ny, nx, width=32, layers=4, modes_x=24, modes_y=24, max_batch=4, seed=0, device=0,
                 stream=None):
        cfg = mm_fno_cfg(width, layers, modes_x, modes_y, max_batch, seed)
        h = C.c_void_p()
        _check(mm_fno_create(C.byref(h), ny, nx, C.byref(cfg), device, stream))
        self.h = h
        self.shape = (ny, nx)
        self.cfg = dict(width=width, layers=layers, modes_x=modes_x, modes_y=modes_y)

    def close(self):
        if self.h:
            mm_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nparams(self):
        return mm_fno_param_count(self.h)

    def get_params(self):
        out = np.zeros(self.nparams(), dtype=np.float32)
        _check(mm_fno_get_params(self.h, _ptr(out), out.size))
        return out

    def set_params(self, p):
        a = np.ascontiguousarray(p, dtype=np.float32)
        _check(mm_fno_set_params(self.h, _ptr(a), a.size))

    def forward(self, u_dev, y_dev, S):
        _check(mm_fno_forward(self.h, C.c_void_p(u_dev.data_ptr()), C.c_void_p(y_dev.data_ptr()), S))

    def grad(self, u_dev, y_dev, S):
        g = np.zeros(self.nparams(), dtype=np.float32)
        loss = C.c_double()
        _check(mm_fno_grad(self.h, C.c_void_p(u_dev.data_ptr()), C.c_void_p(y_dev.data_ptr()), S, _ptr(g),
                           C.byref(loss)))
        return g, loss.value

    def train_step(self, u_dev, y_dev, S, lr):
        loss = C.c_double()
        _check(mm_fno_train_step(self.h, C.c_void_p(u_dev.data_ptr()), C.c_void_p(y_dev.data_ptr()), S, lr,
                                 C.byref(loss)))
        return loss.value
