"""Thin Python binding of the GB300 SF-QED step library (include/qed.h).

Argument marshalling only: every step of the hot path runs in the CUDA kernels of
``libqed_gb300.so``.  PyTorch provides device memory and streams.  If the shared
library has not been built, importing the binding's functions raises -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqed_gb300.so")

QED_OK, QED_ERR_INVALID_ARG, QED_ERR_CUDA, QED_ERR_CAPACITY = 0, 1, 2, 3
QED_ERR_NOT_INITIALIZED, QED_ERR_TIMEOUT, QED_WARN_TABLE_RANGE = 4, 5, 6
QED_ELECTRON, QED_POSITRON, QED_PHOTON = 0, 1, 2
QED_PREC_F64, QED_PREC_MIXED = 0, 1
QED_F_NCS, QED_F_NBW, QED_F_VB, QED_F_SPIN, QED_F_NO_RECOIL, QED_F_DROP_PHOTONS = 1, 2, 4, 8, 16, 32
QED_F_MLP = 64
QED_F_LL, QED_F_MLL, QED_F_MBMT = 128, 256, 512
QED_F_DEPOSIT = 1024
QED_F_BREMS, QED_F_BH = 2048, 4096
QED_FDTD_B, QED_FDTD_E = 0, 1
QED_STATUS_CAPACITY, QED_STATUS_TIMEOUT, QED_STATUS_TABLE_RANGE, QED_STATUS_LOG_FULL = 1, 2, 4, 8
QED_STATUS_SHARD = 16
FIELD_KIND = {"none": 0, "uniform": 1, "plane": 2, "gauss": 3, "grid2d": 4}

ABI_FUNCTIONS = ("qed_init_tables", "qed_destroy", "particles_create", "particles_count",
                 "particles_set_count", "particles_destroy", "qed_set_next_id", "qed_get_next_id",
                 "qed_step", "qed_step_host", "qed_step_static", "qed_step_begin", "qed_step_end",
                 "qed_read_status", "qed_copy_table",
                 "qed_set_timing", "qed_get_timing", "qed_diag", "qed_ctx_share", "qed_batch_create",
                 "qed_batch_step", "qed_batch_run", "qed_batch_clock", "qed_batch_get_config",
                 "qed_batch_set_config", "qed_batch_tune", "qed_batch_destroy", "qed_mlp_train",
                 "qed_mlp_set_params", "qed_mlp_get_params", "qed_mlp_eval", "qed_mlp_target", "qed_fdtd_advance",
                 "qed_sort_cells", "qed_philox_blocks", "qed_set_medium", "qed_copy_medium_table",
                 "qed_last_error")
MLP_PARAMS = 4481
QED_DIAG_SPECTRUM, QED_DIAG_DETECTOR = 0, 1


class qed_soa(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("x", "y", "z", "px", "py", "pz", "s1", "s2", "s3", "theta", "w")] + [
        ("id", C.c_void_p)]


class qed_fields(C.Structure):
    _fields_ = [("kind", C.c_int), ("circular", C.c_int), ("a0", C.c_double), ("phi0", C.c_double),
                ("len", C.c_double), ("w0", C.c_double), ("zf", C.c_double), ("E", C.c_double * 3),
                ("B", C.c_double * 3), ("gEx", C.c_void_p), ("gEy", C.c_void_p), ("gEz", C.c_void_p),
                ("gBx", C.c_void_p), ("gBy", C.c_void_p), ("gBz", C.c_void_p), ("nx", C.c_int),
                ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double), ("x0", C.c_double),
                ("y0", C.c_double), ("periodic", C.c_int), ("gJx", C.c_void_p), ("gJy", C.c_void_p),
                ("gJz", C.c_void_p)]


class qed_grid2d(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz")] + [
        ("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double), ("periodic", C.c_int)]


class qed_step_stats(C.Structure):
    _fields_ = [("n_ncs", C.c_uint64 * 2), ("n_nbw", C.c_uint64), ("n_range", C.c_uint64),
                ("n_drop", C.c_uint64), ("n_steps", C.c_uint64), ("n_processed", C.c_uint64),
                ("n_coarse", C.c_uint64), ("n_brems", C.c_uint64 * 2), ("n_bh", C.c_uint64)]


class qed_medium(C.Structure):
    _fields_ = [("Z", C.c_int), ("n", C.c_double), ("k_min", C.c_double), ("axis", C.c_int),
                ("lo", C.c_double), ("hi", C.c_double)]


class qed_diag_spec(C.Structure):
    _fields_ = [("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("lo_x", C.c_double), ("hi_x", C.c_double),
                ("lo_y", C.c_double), ("hi_y", C.c_double), ("ref", C.c_double * 3)]


class qed_ensemble(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("e", C.c_void_p), ("pos", C.c_void_p), ("ph", C.c_void_p),
                ("fields", qed_fields), ("t0", C.c_double), ("step0", C.c_uint32), ("seed", C.c_uint64),
                ("dev_stats", C.c_void_p)]


class qed_batch_config(C.Structure):
    _fields_ = [("stream_blocks_per_sm", C.c_int), ("event_blocks_per_sm", C.c_int), ("smem_rates", C.c_int)]


class QedError(RuntimeError):
    pass


_lib = None


def lib():
    """Load libqed_gb300.so (built by ``build()``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise QedError(f"{LIB_PATH} is missing: run paper_2306_11288_gb300.build()")
        L = C.CDLL(LIB_PATH)
        vp, u64, u32, d = C.c_void_p, C.c_uint64, C.c_uint32, C.c_double
        L.qed_init_tables.argtypes = [C.POINTER(vp), vp]
        L.qed_destroy.argtypes = [vp]
        L.particles_create.argtypes = [vp, C.c_int, C.POINTER(qed_soa), u64, u64, C.c_int, vp, C.POINTER(vp)]
        L.particles_count.argtypes = [vp, C.POINTER(u64), vp]
        L.particles_set_count.argtypes = [vp, u64, vp]
        L.particles_destroy.argtypes = [vp]
        L.qed_set_next_id.argtypes = [vp, u64, vp]
        L.qed_get_next_id.argtypes = [vp, C.POINTER(u64), vp]
        L.qed_step.argtypes = [vp, vp, vp, vp, C.POINTER(qed_fields), d, d, u64, u32, u32, vp, vp]
        L.qed_step_host.argtypes = [vp, vp, vp, vp, C.POINTER(qed_soa), C.POINTER(qed_soa),
                                    C.POINTER(qed_soa), C.POINTER(u64), C.POINTER(qed_fields), d, d, u64,
                                    u32, u32, vp]
        L.qed_step_static.argtypes = [vp, vp, vp, vp, C.POINTER(qed_fields), d, d, u64, u32, u32, vp, vp]
        L.qed_step_begin.argtypes = [vp, vp, vp, vp, C.POINTER(qed_fields), d, d, u64, u32, u32, vp, vp, vp]
        L.qed_step_end.argtypes = [vp, vp, C.c_int, C.c_int, vp]
        L.qed_read_status.argtypes = [vp, C.POINTER(u32), C.c_int, vp]
        L.qed_copy_table.argtypes = [vp, C.c_int, C.POINTER(C.c_double), u64, C.POINTER(u64), vp]
        L.qed_philox_blocks.argtypes = [vp, u64, vp, u64, vp]
        L.qed_set_timing.argtypes = [vp, C.c_int]
        L.qed_get_timing.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(u64)]
        L.qed_diag.argtypes = [vp, vp, C.POINTER(qed_diag_spec), vp, vp]
        L.qed_ctx_share.argtypes = [vp, vp, C.POINTER(vp)]
        L.qed_batch_create.argtypes = [vp, C.POINTER(qed_ensemble), C.c_int, d, u32, vp, C.POINTER(vp)]
        L.qed_batch_step.argtypes = [vp, vp]
        L.qed_batch_run.argtypes = [vp, u32, vp]
        L.qed_batch_clock.argtypes = [vp, C.c_int, C.POINTER(d), C.POINTER(u32), vp]
        L.qed_batch_get_config.argtypes = [vp, C.POINTER(qed_batch_config)]
        L.qed_batch_set_config.argtypes = [vp, C.POINTER(qed_batch_config)]
        L.qed_batch_tune.argtypes = [vp, u32, vp, C.POINTER(qed_batch_config), C.POINTER(d)]
        L.qed_batch_destroy.argtypes = [vp]
        L.qed_mlp_train.argtypes = [vp, u64, u32, u64, vp]
        L.qed_mlp_set_params.argtypes = [vp, C.POINTER(C.c_float), vp]
        L.qed_mlp_get_params.argtypes = [vp, C.POINTER(C.c_float), vp]
        L.qed_mlp_eval.argtypes = [vp, vp, vp, u64, vp]
        L.qed_mlp_target.argtypes = [vp, vp, vp, u64, vp]
        L.qed_fdtd_advance.argtypes = [C.POINTER(qed_grid2d), C.c_int, d, vp]
        L.qed_sort_cells.argtypes = [vp, vp, C.POINTER(qed_fields), vp]
        L.qed_set_medium.argtypes = [vp, C.POINTER(qed_medium), vp]
        L.qed_copy_medium_table.argtypes = [vp, C.POINTER(C.c_double), u64, C.POINTER(u64), vp]
        L.qed_last_error.restype = C.c_char_p
        for name in ABI_FUNCTIONS:
            if name != "qed_last_error":
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def _check(rc: int, what: str):
    if rc != QED_OK:
        msg = lib().qed_last_error().decode(errors="replace")
        raise QedError(f"{what} failed with status {rc}: {msg}")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream)


# ---- the C-ABI calls, same names -------------------------------------------------------
def qed_init_tables(stream=None):
    h = C.c_void_p()
    _check(lib().qed_init_tables(C.byref(h), _stream(stream)), "qed_init_tables")
    return h


def qed_destroy(ctx):
    _check(lib().qed_destroy(ctx), "qed_destroy")


def qed_ctx_share(parent, stream=None):
    h = C.c_void_p()
    _check(lib().qed_ctx_share(parent, _stream(stream), C.byref(h)), "qed_ctx_share")
    return h


def qed_batch_create(ctx, ens, dt, flags, stream=None):
    arr = (qed_ensemble * len(ens))(*ens)
    h = C.c_void_p()
    _check(lib().qed_batch_create(ctx, arr, len(ens), float(dt), int(flags), _stream(stream), C.byref(h)),
           "qed_batch_create")
    return h


def qed_batch_step(b, stream=None):
    _check(lib().qed_batch_step(b, _stream(stream)), "qed_batch_step")


def qed_batch_run(b, nsteps, stream=None):
    _check(lib().qed_batch_run(b, int(nsteps), _stream(stream)), "qed_batch_run")


def qed_batch_clock(b, e, stream=None):
    t, st = C.c_double(), C.c_uint32()
    _check(lib().qed_batch_clock(b, int(e), C.byref(t), C.byref(st), _stream(stream)), "qed_batch_clock")
    return float(t.value), int(st.value)


def qed_batch_get_config(b) -> dict:
    c = qed_batch_config()
    _check(lib().qed_batch_get_config(b, C.byref(c)), "qed_batch_get_config")
    return {"stream_blocks_per_sm": c.stream_blocks_per_sm, "event_blocks_per_sm": c.event_blocks_per_sm,
            "smem_rates": c.smem_rates}


def qed_batch_set_config(b, stream_blocks_per_sm, event_blocks_per_sm, smem_rates):
    c = qed_batch_config(int(stream_blocks_per_sm), int(event_blocks_per_sm), int(smem_rates))
    _check(lib().qed_batch_set_config(b, C.byref(c)), "qed_batch_set_config")


def qed_batch_tune(b, steps_per_candidate, stream=None):
    """(chosen launch shape, its particle-steps per second)"""
    c, rate = qed_batch_config(), C.c_double()
    _check(lib().qed_batch_tune(b, int(steps_per_candidate), _stream(stream), C.byref(c), C.byref(rate)),
           "qed_batch_tune")
    return {"stream_blocks_per_sm": c.stream_blocks_per_sm, "event_blocks_per_sm": c.event_blocks_per_sm,
            "smem_rates": c.smem_rates}, float(rate.value)


def qed_mlp_train(ctx, n_samples, batch=1024, seed=1, stream=None):
    _check(lib().qed_mlp_train(ctx, int(n_samples), int(batch), int(seed), _stream(stream)), "qed_mlp_train")


def qed_mlp_set_params(ctx, params, stream=None):
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != MLP_PARAMS:
        raise ValueError(f"expected {MLP_PARAMS} parameters")
    _check(lib().qed_mlp_set_params(ctx, a.ctypes.data_as(C.POINTER(C.c_float)), _stream(stream)),
           "qed_mlp_set_params")


def qed_mlp_get_params(ctx, stream=None) -> np.ndarray:
    a = np.zeros(MLP_PARAMS, dtype=np.float32)
    _check(lib().qed_mlp_get_params(ctx, a.ctypes.data_as(C.POINTER(C.c_float)), _stream(stream)),
           "qed_mlp_get_params")
    return a


def qed_mlp_eval(ctx, dev_in_ptr, dev_out_ptr, n, stream=None):
    _check(lib().qed_mlp_eval(ctx, C.c_void_p(dev_in_ptr), C.c_void_p(dev_out_ptr), int(n), _stream(stream)),
           "qed_mlp_eval")


def qed_mlp_target(ctx, dev_in_ptr, dev_out_ptr, n, stream=None):
    _check(lib().qed_mlp_target(ctx, C.c_void_p(dev_in_ptr), C.c_void_p(dev_out_ptr), int(n), _stream(stream)),
           "qed_mlp_target")


def mlp_apply(ctx, rows: np.ndarray, which="eval") -> np.ndarray:
    """ln u for host rows (ln chi_e, s, r) [n, 3] via the learned sampler ("eval") or the
    table sampler's mixture inverse ("target")."""
    import torch
    x = torch.as_tensor(np.ascontiguousarray(rows, dtype=np.float32), device="cuda")
    y = torch.empty(len(rows), dtype=torch.float32, device="cuda")
    (qed_mlp_eval if which == "eval" else qed_mlp_target)(ctx, x.data_ptr(), y.data_ptr(), len(rows))
    return y.cpu().numpy().astype(np.float64)


def qed_batch_destroy(b):
    _check(lib().qed_batch_destroy(b), "qed_batch_destroy")


def particles_create(ctx, species, soa: qed_soa, n, cap, prec, stream=None):
    h = C.c_void_p()
    _check(lib().particles_create(ctx, int(species), C.byref(soa), int(n), int(cap), int(prec),
                                  _stream(stream), C.byref(h)), "particles_create")
    return h


def particles_count(p, stream=None) -> int:
    v = C.c_uint64()
    _check(lib().particles_count(p, C.byref(v), _stream(stream)), "particles_count")
    return int(v.value)


def particles_set_count(p, n, stream=None):
    _check(lib().particles_set_count(p, int(n), _stream(stream)), "particles_set_count")


def particles_destroy(p):
    _check(lib().particles_destroy(p), "particles_destroy")


def qed_set_next_id(ctx, i, stream=None):
    _check(lib().qed_set_next_id(ctx, int(i), _stream(stream)), "qed_set_next_id")


def qed_get_next_id(ctx, stream=None) -> int:
    v = C.c_uint64()
    _check(lib().qed_get_next_id(ctx, C.byref(v), _stream(stream)), "qed_get_next_id")
    return int(v.value)


def qed_step(ctx, e, pos, ph, fields: qed_fields, t, dt, seed, step, flags, dev_stats=None, stream=None):
    _check(lib().qed_step(ctx, e, pos, ph, C.byref(fields), float(t), float(dt), int(seed), int(step),
                          int(flags), dev_stats, _stream(stream)), "qed_step")


def qed_step_begin(ctx, e, pos, ph, fields: qed_fields, t, dt, seed, step, flags, dev_counts, dev_stats=None,
                   stream=None):
    """First half of a sharded step: writes this rank's (pairs, e- emissions, e+ emissions)
    to dev_counts (device pointer to 3 uint64)."""
    _check(lib().qed_step_begin(ctx, e, pos, ph, C.byref(fields), float(t), float(dt), int(seed), int(step),
                                int(flags), dev_stats, dev_counts, _stream(stream)), "qed_step_begin")


def qed_step_end(ctx, dev_all, rank, world, stream=None):
    """Second half: births numbered after the ranks before ``rank`` (dev_all: device pointer
    to world x 3 uint64, every rank's counts, rank-major)."""
    _check(lib().qed_step_end(ctx, dev_all, int(rank), int(world), _stream(stream)), "qed_step_end")


def qed_step_static(ctx, e, pos, ph, fields: qed_fields, t, dt, seed, step, flags, dev_stats=None, stream=None):
    """qed_step with its scratch in the library's static device array (no allocation);
    particle sets of capacity <= 65536 per species."""
    _check(lib().qed_step_static(ctx, e, pos, ph, C.byref(fields), float(t), float(dt), int(seed), int(step),
                                 int(flags), dev_stats, _stream(stream)), "qed_step_static")


def qed_step_host(ctx, e, pos, ph, host_e, host_pos, host_ph, n_host, fields, t, dt, seed, step, flags,
                  stream=None):
    arr = (C.c_uint64 * 3)(*[int(v) for v in n_host])
    _check(lib().qed_step_host(ctx, e, pos, ph, C.byref(host_e) if host_e else None,
                               C.byref(host_pos) if host_pos else None, C.byref(host_ph) if host_ph else None,
                               arr, C.byref(fields), float(t), float(dt), int(seed), int(step), int(flags),
                               _stream(stream)), "qed_step_host")
    return [int(v) for v in arr]


def qed_read_status(ctx, clear=False, stream=None) -> int:
    v = C.c_uint32()
    _check(lib().qed_read_status(ctx, C.byref(v), int(bool(clear)), _stream(stream)), "qed_read_status")
    return int(v.value)


def qed_copy_table(ctx, which, stream=None) -> np.ndarray:
    n = C.c_uint64()
    _check(lib().qed_copy_table(ctx, int(which), None, 0, C.byref(n), _stream(stream)), "qed_copy_table")
    out = np.zeros(n.value)
    _check(lib().qed_copy_table(ctx, int(which), out.ctypes.data_as(C.POINTER(C.c_double)), n.value,
                                C.byref(n), _stream(stream)), "qed_copy_table")
    return out


def qed_philox_blocks(ctr, key, out, stream=None):
    """Philox4x32-10 on the device for the counters ctr (int32 CUDA tensor, n x 4) under the
    64-bit key; out (int32 CUDA tensor, n x 8) receives per block the words of the kernel-side
    key schedule form, then those of the host-precomputed form (argument marshalling only)."""
    n = ctr.shape[0] if ctr.dim() == 2 else 0
    if ctr.dim() != 2 or ctr.shape[1] != 4 or out.dim() != 2 or out.shape[0] != n or out.shape[1] != 8:
        raise ValueError("qed_philox_blocks: ctr must be n x 4 and out n x 8")
    for tns in (ctr, out):
        if not tns.is_contiguous() or tns.element_size() != 4 or not tns.is_cuda:
            raise ValueError("qed_philox_blocks: contiguous 32-bit CUDA tensors required")
    _check(lib().qed_philox_blocks(C.c_void_p(ctr.data_ptr()), C.c_uint64(int(key) & (2**64 - 1)),
                                   C.c_void_p(out.data_ptr()), C.c_uint64(n), _stream(stream)),
           "qed_philox_blocks")


def diag_spec(kind, nx, ny=1, lo_x=1.0, hi_x=2.0, lo_y=0.0, hi_y=1.0, ref=(0.0, 0.0, 0.0)) -> qed_diag_spec:
    sp = qed_diag_spec()
    sp.kind, sp.nx, sp.ny = int(kind), int(nx), int(ny)
    sp.lo_x, sp.hi_x, sp.lo_y, sp.hi_y = float(lo_x), float(hi_x), float(lo_y), float(hi_y)
    for k in range(3):
        sp.ref[k] = float(ref[k])
    return sp


def qed_diag(ctx, handle, spec: qed_diag_spec, dev_out_ptr: int, stream=None):
    _check(lib().qed_diag(ctx, handle, C.byref(spec), C.c_void_p(dev_out_ptr), _stream(stream)), "qed_diag")


def diag(species: "Species", spec: qed_diag_spec, stream=None) -> dict:
    """Histogram of one device set (see qed_diag): returns bins [ny, nx, 5] (sum w, sum w o1..o3,
    count), total [5], below, above."""
    import torch
    nb = spec.nx * spec.ny
    out = torch.zeros(5 * (nb + 1) + 2, dtype=torch.float64, device="cuda")
    qed_diag(species.ctx, species.handle, spec, out.data_ptr(), stream)
    v = out.cpu().numpy()
    return {"bins": v[:5 * nb].reshape(spec.ny, spec.nx, 5), "total": v[5 * nb:5 * nb + 5],
            "below": float(v[5 * nb + 5]), "above": float(v[5 * nb + 6])}


def qed_set_timing(ctx, enable: bool):
    _check(lib().qed_set_timing(ctx, int(bool(enable))), "qed_set_timing")


def qed_get_timing(ctx):
    """(milliseconds of [photon pass, lepton pass, event kernels], steps timed)"""
    ms = (C.c_double * 3)()
    n = C.c_uint64()
    _check(lib().qed_get_timing(ctx, ms, C.byref(n)), "qed_get_timing")
    return [ms[0], ms[1], ms[2]], int(n.value)


def qed_last_error() -> str:
    return lib().qed_last_error().decode(errors="replace")


# ---- memory plumbing (torch tensors as storage) ----------------------------------------------
_NAMES = ("x", "y", "z", "px", "py", "pz", "s1", "s2", "s3", "theta", "w")


class Species:
    """Device SoA (torch tensors) for one species, wrapped as a qed_particles handle."""

    def __init__(self, ctx, species, cap, prec=QED_PREC_F64, device="cuda", pin_host=False):
        import torch
        self.torch = torch
        self.ctx, self.species, self.cap, self.prec = ctx, species, int(cap), prec
        rt = torch.float64 if prec == QED_PREC_F64 else torch.float32
        self.t = {}
        for k in _NAMES:
            if k == "theta" and species != QED_PHOTON:
                continue
            dt = torch.float64 if k in ("x", "y", "z") else rt
            self.t[k] = torch.zeros(max(self.cap, 1), dtype=dt, device=device)
        self.t["id"] = torch.zeros(max(self.cap, 1), dtype=torch.int64, device=device)
        self.soa = qed_soa()
        for k, v in self.t.items():
            setattr(self.soa, k, v.data_ptr())
        self.handle = particles_create(ctx, species, self.soa, 0, self.cap, prec)
        self._closed = False

    def load(self, d: dict, stream=None):
        n = len(d["id"])
        if n > self.cap:
            raise ValueError("more particles than capacity")
        for k, v in self.t.items():
            if k == "id":
                src = np.asarray(d["id"], dtype=np.uint64).view(np.int64)
            elif k in d:
                src = np.asarray(d[k], dtype=np.float64)
            else:
                continue
            if n:
                v[:n].copy_(self.torch.from_numpy(np.ascontiguousarray(src)).to(v.dtype))
        self.torch.cuda.synchronize()
        particles_set_count(self.handle, n, stream)
        return self

    def count(self, stream=None) -> int:
        return particles_count(self.handle, stream)

    def to_dict(self) -> dict:
        n = self.count()
        out = {}
        for k, v in self.t.items():
            a = v[:n].cpu().numpy()
            out[k] = a.view(np.uint64) if k == "id" else a.astype(np.float64)
        return out

    def close(self):
        if not self._closed:
            self._closed = True
            particles_destroy(self.handle)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fields_from_spec(spec: dict, grid=None) -> qed_fields:
    """Field descriptor dict -> qed_fields; grid components must be CUDA float32 tensors."""
    f = qed_fields()
    f.kind = FIELD_KIND[spec["kind"]]
    f.circular = int(spec.get("circular", 0))
    f.a0 = float(spec.get("a0", 0.0))
    f.phi0 = float(spec.get("phi0", 0.0))
    f.len = float(spec.get("len", 1.0))
    f.w0 = float(spec.get("w0", 1.0))
    f.zf = float(spec.get("zf", 0.0))
    f.E[:] = [float(v) for v in spec.get("E", (0, 0, 0))]
    f.B[:] = [float(v) for v in spec.get("B", (0, 0, 0))]
    if grid is not None:
        for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
            setattr(f, "g" + k, grid[k].data_ptr())
        f.ny, f.nx = grid["Ey"].shape
        f.dx, f.dy = float(grid["dx"]), float(grid["dy"])
        f.x0, f.y0 = float(grid.get("x0", 0.0)), float(grid.get("y0", 0.0))
        f.periodic = int(grid.get("periodic", 0))
        for k in ("Jx", "Jy", "Jz"):
            if k in grid:
                setattr(f, "g" + k, grid[k].data_ptr())
    return f


def qed_set_medium(ctx, medium, stream=None):
    """medium: dict(Z, n, k_min, axis, lo, hi) (Sec. III E matter) or None to remove it."""
    if medium is None:
        _check(lib().qed_set_medium(ctx, None, _stream(stream)), "qed_set_medium")
        return
    m = qed_medium(int(medium["Z"]), float(medium["n"]), float(medium["k_min"]), int(medium.get("axis", 2)),
                   float(medium.get("lo", -1e300)), float(medium.get("hi", 1e300)))
    _check(lib().qed_set_medium(ctx, C.byref(m), _stream(stream)), "qed_set_medium")


def qed_copy_medium_table(ctx, stream=None):
    import numpy as np
    n = C.c_uint64()
    _check(lib().qed_copy_medium_table(ctx, None, 0, C.byref(n), _stream(stream)), "qed_copy_medium_table")
    out = np.zeros(n.value)
    _check(lib().qed_copy_medium_table(ctx, out.ctypes.data_as(C.POINTER(C.c_double)), n.value, C.byref(n),
                                       _stream(stream)), "qed_copy_medium_table")
    return out


def qed_sort_cells(ctx, handle, grid: qed_fields, stream=None):
    _check(lib().qed_sort_cells(ctx, handle, C.byref(grid), _stream(stream)), "qed_sort_cells")


def qed_fdtd_advance(g: qed_grid2d, which, dt, stream=None):
    _check(lib().qed_fdtd_advance(C.byref(g), int(which), float(dt), _stream(stream)), "qed_fdtd_advance")


class Simulation:
    """One context + e-, e+, photon sets stepping together (device resident)."""

    def __init__(self, wl: dict, prec=QED_PREC_F64, cap_e=None, cap_p=None, cap_ph=None, ctx=None):
        import torch
        self.torch = torch
        self.ctx = ctx if ctx is not None else qed_init_tables()
        self.own_ctx = ctx is None
        ne, npos, nph = len(wl["e"]["id"]), len(wl["pos"]["id"]), len(wl["ph"]["id"])
        self.e = Species(self.ctx, QED_ELECTRON, cap_e if cap_e is not None else max(4 * (ne + nph), 16),
                         prec).load(wl["e"])
        self.pos = Species(self.ctx, QED_POSITRON, cap_p if cap_p is not None else max(4 * (ne + npos + nph), 16),
                           prec).load(wl["pos"])
        self.ph = Species(self.ctx, QED_PHOTON, cap_ph if cap_ph is not None else max(8 * (ne + npos + nph), 16),
                          prec).load(wl["ph"])
        self.grid = None
        if wl["field"]["kind"] == "grid2d":
            g = wl["grid"]
            self.grid = {k: torch.as_tensor(np.ascontiguousarray(g[k]), dtype=torch.float32, device="cuda")
                         for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")}
            self.grid.update({k: g[k] for k in ("dx", "dy") if k in g})
            self.grid.update({k: g.get(k, 0.0) for k in ("x0", "y0")})
            self.grid["periodic"] = int(g.get("periodic", 0))
        self.fields = fields_from_spec(wl["field"], self.grid)
        self.dt = float(wl["dt"])
        self.t = float(wl.get("t0", 0.0))
        self.seed = int(wl["seed"])
        self.step_no = int(wl.get("step0", 0))
        self.stats = torch.zeros(11, dtype=torch.int64, device="cuda")
        qed_set_next_id(self.ctx, int(wl["next_id"]))
        if wl.get("medium") is not None:
            qed_set_medium(self.ctx, wl["medium"])
        qed_read_status(self.ctx, clear=True)

    def run(self, nsteps, flags, stream=None):
        for _ in range(nsteps):
            qed_step(self.ctx, self.e.handle, self.pos.handle, self.ph.handle, self.fields, self.t, self.dt,
                     self.seed, self.step_no, flags, self.stats.data_ptr(), stream)
            self.t += self.dt
            self.step_no += 1

    def step_begin(self, flags, stream=None):
        """qed_step_begin of the next step; returns this rank's counts (3, int64, device)."""
        torch = self.torch
        self._counts = torch.zeros(3, dtype=torch.int64, device="cuda")
        qed_step_begin(self.ctx, self.e.handle, self.pos.handle, self.ph.handle, self.fields, self.t, self.dt,
                       self.seed, self.step_no, flags, self._counts.data_ptr(), self.stats.data_ptr(), stream)
        return self._counts

    def step_end(self, all_counts, rank, world, stream=None):
        """qed_step_end with every rank's counts (world x 3 int64 tensor, rank-major)."""
        torch = self.torch
        allc = all_counts.to(device="cuda", dtype=torch.int64).contiguous()
        if allc.numel() != 3 * world:
            raise ValueError("all_counts must hold world x 3 counts")
        self._all = allc   # kept alive until the step has run
        qed_step_end(self.ctx, allc.data_ptr(), rank, world, stream)
        self.t += self.dt
        self.step_no += 1

    def state(self) -> dict:
        self.torch.cuda.synchronize()
        return {"e": self.e.to_dict(), "pos": self.pos.to_dict(), "ph": self.ph.to_dict(),
                "next_id": qed_get_next_id(self.ctx)}

    def counters(self) -> dict:
        s = self.stats.cpu().numpy()
        return {"n_ncs_e": int(s[0]), "n_ncs_p": int(s[1]), "n_nbw": int(s[2]), "n_range": int(s[3]),
                "n_drop": int(s[4]), "n_steps": int(s[5]), "n_processed": int(s[6]), "n_coarse": int(s[7]),
                "n_brems_e": int(s[8]), "n_brems_p": int(s[9]), "n_bh": int(s[10])}

    def status(self, clear=False) -> int:
        return qed_read_status(self.ctx, clear)

    def close(self):
        for s in (self.e, self.pos, self.ph):
            s.close()
        if self.own_ctx:
            qed_destroy(self.ctx)


class Batch:
    """Independent ensembles stepped together (qed_batch_*): one Simulation per workload,
    each on a context sharing `ctx`'s tables.  All workloads must share dt."""

    def __init__(self, wls: list, prec=QED_PREC_F64, flags=None, ctx=None, caps=None):
        import torch
        self.torch = torch
        self.ctx = ctx if ctx is not None else qed_init_tables()
        self.own_ctx = ctx is None
        dts = {float(w["dt"]) for w in wls}
        if len(dts) != 1:
            raise ValueError("all ensembles of a batch share dt")
        self.dt = dts.pop()
        self.flags = (QED_F_NCS | QED_F_NBW | QED_F_VB | QED_F_SPIN) if flags is None else flags
        caps = caps or [{}] * len(wls)
        self.sims = [Simulation(w, prec=prec, ctx=qed_ctx_share(self.ctx), **c) for w, c in zip(wls, caps)]
        ens = []
        for s in self.sims:
            ens.append(qed_ensemble(s.ctx, s.e.handle, s.pos.handle, s.ph.handle, s.fields, s.t, s.step_no, s.seed,
                                    s.stats.data_ptr()))
        torch.cuda.synchronize()
        self.b = qed_batch_create(self.ctx, ens, self.dt, self.flags)

    def step(self, n=1, stream=None):
        for _ in range(n):
            qed_batch_step(self.b, stream)

    def run(self, n, stream=None):
        qed_batch_run(self.b, n, stream)

    def clocks(self):
        return [qed_batch_clock(self.b, e) for e in range(len(self.sims))]

    def close(self):
        if self.b is not None:
            qed_batch_destroy(self.b)
            self.b = None
        for s in self.sims:
            c = s.ctx
            s.close()
            qed_destroy(c)
        self.sims = []
        if self.own_ctx:
            qed_destroy(self.ctx)
            self.own_ctx = False


class PicSimulation(Simulation):
    """The step inside the PIC loop of Sec. II F on a 2D3V Yee grid of the library: E^n and
    B^{n-1/2} stored in float device tensors; per step FDTD_B(dt/2), qed_step with
    QED_F_DEPOSIT (gathers E^n, B^n; deposits J^{n+1/2}), FDTD_B(dt/2), FDTD_E(dt) (which
    consumes J and clears it).  `fields` (optional) gives initial E, B arrays [ny][nx]."""

    def __init__(self, wl: dict, nx, ny, dx, dy, periodic=1, fields=None, x0=0.0, y0=0.0, prec=QED_PREC_F64,
                 **caps):
        import torch
        self.yee = {k: torch.zeros((ny, nx), dtype=torch.float32, device="cuda")
                    for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz")}
        for k, v in (fields or {}).items():
            self.yee[k].copy_(torch.as_tensor(np.asarray(v, dtype=np.float32)))
        # the particle sets and context; the field descriptor is set to the Yee grid below
        super().__init__(dict(wl, field={"kind": "none"}), prec=prec, **caps)
        grid = dict(self.yee)
        grid.update({"dx": dx, "dy": dy, "x0": x0, "y0": y0, "periodic": periodic})
        self.grid = grid
        self.fields = fields_from_spec({"kind": "grid2d"}, grid)
        self.g = qed_grid2d()
        for k, v in self.yee.items():
            setattr(self.g, k, v.data_ptr())
        self.g.nx, self.g.ny, self.g.dx, self.g.dy, self.g.periodic = nx, ny, float(dx), float(dy), int(periodic)

    def run(self, nsteps, flags, stream=None):
        for _ in range(nsteps):
            qed_fdtd_advance(self.g, QED_FDTD_B, 0.5 * self.dt, stream)
            qed_step(self.ctx, self.e.handle, self.pos.handle, self.ph.handle, self.fields, self.t, self.dt,
                     self.seed, self.step_no, flags | QED_F_DEPOSIT, self.stats.data_ptr(), stream)
            qed_fdtd_advance(self.g, QED_FDTD_B, 0.5 * self.dt, stream)
            qed_fdtd_advance(self.g, QED_FDTD_E, self.dt, stream)
            self.t += self.dt
            self.step_no += 1

    def field_arrays(self) -> dict:
        self.torch.cuda.synchronize()
        return {k: v.cpu().numpy().astype(np.float64) for k, v in self.yee.items()}


# ---------------------------------------------------------------------------------
# Several ranks (one process per GPU) stepping one population, each its own part.  The
# step's only exchange is the births' id numbering (one all-gather of 3 counts per rank);
# diagnostics are summed over the ranks at the end (one all-reduce).
# ---------------------------------------------------------------------------------
def shard_exchange(counts, group=None):
    """Every rank's (pairs, e- emissions, e+ emissions) of this step: an all-gather of
    ``counts`` (3 int64).  With NCCL the tensors stay on the device; with gloo they go
    through host memory.  Returns a (world, 3) tensor on ``counts``' device."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    host = dist.get_backend(group) == "gloo"
    src = counts.detach().to("cpu") if host else counts
    out = [torch.empty_like(src) for _ in range(world)]
    dist.all_gather(out, src, group=group)
    return torch.stack(out).to(counts.device)


def sharded_step(sim, flags, group=None, stream=None):
    """One step of ``sim`` (a Simulation holding this rank's part) with ids numbered across
    the ranks of ``group`` (qed_step_begin, shard_exchange, qed_step_end)."""
    import torch.distributed as dist
    c = sim.step_begin(flags, stream)
    allc = shard_exchange(c, group)
    sim.step_end(allc, dist.get_rank(group), dist.get_world_size(group), stream)


def allreduce_hist(h, group=None):
    """Sum of a histogram (any tensor) over the ranks of ``group``, in place; with gloo
    through host memory.  Returns ``h``."""
    import torch.distributed as dist
    if dist.get_backend(group) == "gloo" and h.device.type != "cpu":
        t = h.detach().cpu()
        dist.all_reduce(t, group=group)
        h.copy_(t)
    else:
        dist.all_reduce(h, group=group)
    return h
