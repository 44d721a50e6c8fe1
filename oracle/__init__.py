"""FP64 CPU oracle of the spin/polarization-resolved SF-QED particle step
(Wan et al., arXiv:2306.11288).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py``.  The product library never imports,
links or calls anything here, and this package shares no code with it.

The C source (``qed_oracle.c``) is compiled with gcc into ``oracle/_build`` on first
use; ``build()`` forces that.  The Python side only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qed_oracle.c")
_HDR = os.path.join(_HERE, "qed_oracle.h")
_OUT = os.path.join(_HERE, "_build", "libqed_oracle.so")
_lock = threading.Lock()
_lib = None

F_NCS, F_NBW, F_VB, F_SPIN, F_NO_RECOIL, F_DROP_PHOTONS = 1, 2, 4, 8, 16, 32
F_LL, F_MLL, F_MBMT = 128, 256, 512   # radiative pusher: LL, quantum-corrected LL, radiative T-BMT
F_DEPOSIT = 1024                      # leptons deposit their current (Esirkepov)
F_BREMS, F_BH = 2048, 4096            # bremsstrahlung, Bethe-Heitler pairs in matter
FIELD_NONE, FIELD_UNIFORM, FIELD_PLANE, FIELD_GAUSS, FIELD_GRID2D = 0, 1, 2, 3, 4
# the decisions of a step, in the near-tie log (qed_oracle.h OR_D_*)
DECISIONS = ("ncs", "ncs_collapse", "ncs_comp", "ncs_spin", "ncs_stokes", "nbw", "nbw_comp", "nbw_spin",
             "brems", "bh")


def build(force: bool = False) -> str:
    """Compile the oracle (plain gcc, -ffp-contract=off) and return the .so path."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    fresh = os.path.exists(_OUT) and os.path.getmtime(_OUT) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not fresh:
        tmp = _OUT + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        # OpenMP (optional: the particle loops of a step across host cores); plain build
        # when the compiler has no OpenMP runtime
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _OUT)
    return _OUT


class Particles(C.Structure):
    _fields_ = [(n, C.POINTER(C.c_double)) for n in
                ("x", "y", "z", "px", "py", "pz", "s1", "s2", "s3", "theta", "w")] + [
        ("id", C.POINTER(C.c_uint64)), ("n", C.c_uint64), ("cap", C.c_uint64)]


class Fields(C.Structure):
    _fields_ = [("kind", C.c_int), ("circular", C.c_int), ("a0", C.c_double),
                ("phi0", C.c_double), ("len", C.c_double), ("w0", C.c_double),
                ("zf", C.c_double), ("E", C.c_double * 3), ("B", C.c_double * 3),
                ("gEx", C.POINTER(C.c_float)), ("gEy", C.POINTER(C.c_float)),
                ("gEz", C.POINTER(C.c_float)), ("gBx", C.POINTER(C.c_float)),
                ("gBy", C.POINTER(C.c_float)), ("gBz", C.POINTER(C.c_float)),
                ("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("periodic", C.c_int),
                ("gJx", C.POINTER(C.c_double)), ("gJy", C.POINTER(C.c_double)), ("gJz", C.POINTER(C.c_double))]


class Grid(C.Structure):
    _fields_ = [(n, C.POINTER(C.c_double)) for n in ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz")] + [
        ("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double), ("periodic", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n_ncs", C.c_uint64 * 2), ("n_nbw", C.c_uint64), ("n_range", C.c_uint64),
                ("n_drop", C.c_uint64), ("n_near", C.c_uint64), ("n_coarse", C.c_uint64),
                ("n_brems", C.c_uint64 * 2), ("n_bh", C.c_uint64)]


class Medium(C.Structure):
    _fields_ = [("Z", C.c_int), ("n", C.c_double), ("k_min", C.c_double), ("axis", C.c_int),
                ("lo", C.c_double), ("hi", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, pd, u64 = C.c_double, C.POINTER(C.c_double), C.c_uint64
            L.or_ctx_create.restype = C.c_void_p
            L.or_ctx_destroy.argtypes = [C.c_void_p]
            L.or_set_next_id.argtypes = [C.c_void_p, u64]
            L.or_get_next_id.argtypes = [C.c_void_p]
            L.or_get_next_id.restype = u64
            L.or_near_log.argtypes = [C.c_void_p, C.POINTER(u64), C.POINTER(C.c_uint32),
                                      C.POINTER(C.c_uint32), pd, u64]
            L.or_near_log.restype = u64
            L.or_set_near_tol.argtypes = [C.c_void_p, d]
            L.or_set_threads.argtypes = [C.c_void_p, C.c_int]
            L.or_set_threads.restype = C.c_int
            L.or_step.argtypes = [C.c_void_p, C.POINTER(Particles), C.POINTER(Particles),
                                  C.POINTER(Particles), C.POINTER(Fields), d, d, u64,
                                  C.c_uint32, C.c_uint32, C.POINTER(Stats)]
            L.or_step_decide.argtypes = [C.c_void_p, C.POINTER(Particles), C.POINTER(Particles),
                                         C.POINTER(Particles), C.POINTER(Fields), d, d, u64,
                                         C.c_uint32, C.c_uint32, C.POINTER(Stats), C.POINTER(u64)]
            L.or_step_commit.argtypes = [C.c_void_p, C.POINTER(Particles), C.POINTER(Particles),
                                         C.POINTER(Particles), C.POINTER(u64), C.POINTER(Stats)]
            L.or_shard_bases.argtypes = [u64, C.POINTER(u64), C.c_int, C.c_int, C.POINTER(u64)]
            L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
            L.or_uniforms.argtypes = [u64, u64, C.c_uint32, C.c_uint32, pd]
            L.or_besselk_scaled.argtypes = [d, pd]
            L.or_ktable.argtypes = [C.c_void_p, d, pd]
            L.or_ncs_rates.argtypes = [C.c_void_p, d, pd]
            L.or_ncs_invcdf.argtypes = [C.c_void_p, C.c_int, d, d]
            L.or_ncs_invcdf.restype = d
            L.or_nbw_rates.argtypes = [C.c_void_p, d, pd]
            L.or_nbw_invcdf.argtypes = [C.c_void_p, C.c_int, d, d]
            L.or_nbw_invcdf.restype = d
            L.or_vb_m.argtypes = [C.c_void_p, d, pd]
            L.or_rr_funcs.argtypes = [C.c_void_p, d, pd]
            L.or_scorer_gi_prime.argtypes = [d]
            L.or_scorer_gi_prime.restype = d
            L.or_field.argtypes = [C.POINTER(Fields), d, d, d, d, pd, pd]
            L.or_ncs_F.argtypes = [C.c_void_p, d, d, pd, pd, pd, pd, pd]
            L.or_nbw_G.argtypes = [C.c_void_p, d, d, d, pd, pd, pd, pd, pd, pd]
            L.or_fdtd_b.argtypes = [C.POINTER(Grid), d]
            L.or_fdtd_e.argtypes = [C.POINTER(Grid), d]
            L.or_charge_tsc.argtypes = [C.POINTER(Grid), d, d, pd, pd, pd, u64, pd]
            L.or_set_medium.argtypes = [C.c_void_p, C.POINTER(Medium)]
            L.or_screening.argtypes = [d, d, pd]
            L.or_coulomb_f.argtypes = [C.c_int]
            L.or_coulomb_f.restype = d
            L.or_brems_D.argtypes = [C.c_int, d, d]
            L.or_brems_D.restype = d
            L.or_pair_D.argtypes = [C.c_int, d, d]
            L.or_pair_D.restype = d
            L.or_medium_sigma.argtypes = [C.c_void_p, C.c_int, d]
            L.or_medium_sigma.restype = d
            L.or_medium_sample.argtypes = [C.c_void_p, C.c_int, d, d]
            L.or_medium_sample.restype = d
            L.or_table.argtypes = [C.c_void_p, C.c_int, C.POINTER(u64)]
            L.or_table.restype = pd
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(v):
    return np.ascontiguousarray(v, dtype=np.float64)


class ParticleArrays:
    """Owned numpy SoA for one species; ``photon`` adds the basis angle."""

    NAMES = ("x", "y", "z", "px", "py", "pz", "s1", "s2", "s3", "theta", "w")

    def __init__(self, cap: int, photon: bool = False):
        self.cap = int(cap)
        self.photon = photon
        self.arr = {k: np.zeros(max(self.cap, 1)) for k in self.NAMES}
        self.id = np.zeros(max(self.cap, 1), dtype=np.uint64)
        self.n = 0
        self._s = Particles()
        for k in self.NAMES:
            setattr(self._s, k, _dp(self.arr[k]) if (photon or k != "theta") else None)
        self._s.id = self.id.ctypes.data_as(C.POINTER(C.c_uint64))
        self._s.cap = self.cap

    def load(self, d: dict):
        n = len(d["id"])
        if n > self.cap:
            raise ValueError("more particles than capacity")
        for k in self.NAMES:
            if k in d:
                self.arr[k][:n] = d[k]
        self.id[:n] = d["id"]
        self.n = n
        return self

    def view(self) -> dict:
        out = {k: self.arr[k][: self.n].copy() for k in self.NAMES if self.photon or k != "theta"}
        out["id"] = self.id[: self.n].copy()
        return out

    def struct(self):
        self._s.n = self.n
        return C.byref(self._s)

    def sync(self):
        self.n = int(self._s.n)


def make_fields(kind=FIELD_NONE, circular=0, a0=0.0, phi0=0.0, length=1.0, w0=1.0, zf=0.0,
                E=(0, 0, 0), B=(0, 0, 0), grid=None):
    f = Fields()
    f.kind, f.circular, f.a0, f.phi0, f.len, f.w0, f.zf = kind, circular, a0, phi0, length, w0, zf
    f.E[:] = list(E)
    f.B[:] = list(B)
    f._keep = None
    if grid is not None:
        comps = [np.ascontiguousarray(grid[k], dtype=np.float32) for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")]
        f._keep = comps
        for name, a in zip(("gEx", "gEy", "gEz", "gBx", "gBy", "gBz"), comps):
            setattr(f, name, a.ctypes.data_as(C.POINTER(C.c_float)))
        f.ny, f.nx = comps[0].shape
        f.dx, f.dy, f.x0, f.y0 = grid["dx"], grid["dy"], grid.get("x0", 0.0), grid.get("y0", 0.0)
        f.periodic = int(grid.get("periodic", 0))
    return f


def _stats_dict(st) -> dict:
    return {"n_ncs_e": st.n_ncs[0], "n_ncs_p": st.n_ncs[1], "n_nbw": st.n_nbw,
            "n_range": st.n_range, "n_drop": st.n_drop, "n_near": st.n_near, "n_coarse": st.n_coarse,
            "n_brems_e": st.n_brems[0], "n_brems_p": st.n_brems[1], "n_bh": st.n_bh}


def shard_bases(next_id: int, all_counts, rank: int) -> np.ndarray:
    """or_shard_bases: the 4 id bases of rank ``rank`` from every rank's 3 counts."""
    a = np.ascontiguousarray(np.asarray(all_counts, dtype=np.uint64).reshape(-1, 3))
    out = np.zeros(4, dtype=np.uint64)
    lib().or_shard_bases(int(next_id), a.ctypes.data_as(C.POINTER(C.c_uint64)), int(rank), int(a.shape[0]),
                         out.ctypes.data_as(C.POINTER(C.c_uint64)))
    return out


class Oracle:
    """Owns one oracle context (tables + id counter)."""

    def __init__(self):
        self.L = lib()
        self.ctx = self.L.or_ctx_create()
        if not self.ctx:
            raise MemoryError("or_ctx_create failed")

    def __del__(self):
        try:
            self.L.or_ctx_destroy(self.ctx)
        except Exception:
            pass

    # --- simulation ---------------------------------------------------------------
    def set_next_id(self, i: int):
        self.L.or_set_next_id(self.ctx, int(i))

    def next_id(self) -> int:
        return int(self.L.or_get_next_id(self.ctx))

    def step(self, e, pos, ph, fields, t, dt, seed, step, flags):
        st = Stats()
        self.L.or_step(self.ctx, e.struct(), pos.struct(), ph.struct(), C.byref(fields),
                       float(t), float(dt), int(seed), int(step), int(flags), C.byref(st))
        e.sync(); pos.sync(); ph.sync()
        return _stats_dict(st)

    def step_decide(self, e, pos, ph, fields, t, dt, seed, step, flags):
        """Every decision of one step; returns (counts, stats): counts = (pairs, e- emissions,
        e+ emissions), held until step_commit."""
        st = Stats()
        cnt = np.zeros(3, dtype=np.uint64)
        self.L.or_step_decide(self.ctx, e.struct(), pos.struct(), ph.struct(), C.byref(fields),
                              float(t), float(dt), int(seed), int(step), int(flags), C.byref(st),
                              cnt.ctypes.data_as(C.POINTER(C.c_uint64)))
        e.sync(); pos.sync(); ph.sync()
        return cnt, _stats_dict(st)

    def step_commit(self, e, pos, ph, bases=None):
        """The births of the decided step, numbered from ``bases`` (4 ids, or_step_commit)."""
        st = Stats()
        b = None
        if bases is not None:
            b = np.ascontiguousarray(bases, dtype=np.uint64)
        r = self.L.or_step_commit(self.ctx, e.struct(), pos.struct(), ph.struct(),
                                  b.ctypes.data_as(C.POINTER(C.c_uint64)) if b is not None else None, C.byref(st))
        if r != 0:
            raise RuntimeError("or_step_commit without a decided step")
        e.sync(); pos.sync(); ph.sync()
        return _stats_dict(st)

    def set_threads(self, n: int) -> int:
        """Threads of the particle loops of a step (OpenMP); returns the count in effect."""
        return int(self.L.or_set_threads(self.ctx, int(n)))

    def set_near_tol(self, tol: float):
        """Log every decision whose draw lies within ``tol`` relative of its threshold."""
        self.L.or_set_near_tol(self.ctx, float(tol))

    def near_log(self, cap=1 << 20):
        """(ids, steps, kinds, margins) of the logged near-tie decisions (kinds: DECISIONS)."""
        ids = np.zeros(cap, dtype=np.uint64)
        steps = np.zeros(cap, dtype=np.uint32)
        kinds = np.zeros(cap, dtype=np.uint32)
        m = np.zeros(cap)
        n = int(self.L.or_near_log(self.ctx, ids.ctypes.data_as(C.POINTER(C.c_uint64)),
                                   steps.ctypes.data_as(C.POINTER(C.c_uint32)),
                                   kinds.ctypes.data_as(C.POINTER(C.c_uint32)), _dp(m), cap))
        if n > cap:
            raise RuntimeError(f"near-tie log overflow: {n} entries, {cap} kept")
        return ids[:n], steps[:n], kinds[:n], m[:n]

    # --- pieces -------------------------------------------------------------------
    def ktable(self, x):
        o = np.zeros(3)
        self.L.or_ktable(self.ctx, float(x), _dp(o))
        return o

    def ncs_rates(self, chi):
        o = np.zeros(2)
        self.L.or_ncs_rates(self.ctx, float(chi), _dp(o))
        return o

    def ncs_invcdf(self, comp, chi, t):
        return self.L.or_ncs_invcdf(self.ctx, int(comp), float(chi), float(t))

    def nbw_rates(self, chig):
        o = np.zeros(2)
        self.L.or_nbw_rates(self.ctx, float(chig), _dp(o))
        return o

    def nbw_invcdf(self, comp, chig, t):
        return self.L.or_nbw_invcdf(self.ctx, int(comp), float(chig), float(t))

    def vb_m(self, chig):
        o = np.zeros(2)
        self.L.or_vb_m(self.ctx, float(chig), _dp(o))
        return o

    def rr_funcs(self, chi):
        """q(chi), psi1, psi2, psi3 of the radiative pusher (Sec. III A, B)"""
        o = np.zeros(4)
        self.L.or_rr_funcs(self.ctx, float(chi), _dp(o))
        return o

    def ncs_F(self, u, chi, n, a, Si, Sf):
        o = np.zeros(4)
        n, a, Si, Sf = map(_vec, (n, a, Si, Sf))
        self.L.or_ncs_F(self.ctx, float(u), float(chi), _dp(n), _dp(a), _dp(Si), _dp(Sf), _dp(o))
        return o

    def nbw_G(self, delta, omega, chig, ap, bp, vp, Sp, Sm):
        o = np.zeros(4)
        ap, bp, vp, Sp, Sm = map(_vec, (ap, bp, vp, Sp, Sm))
        self.L.or_nbw_G(self.ctx, float(delta), float(omega), float(chig), _dp(ap), _dp(bp),
                        _dp(vp), _dp(Sp), _dp(Sm), _dp(o))
        return o

    def set_medium(self, medium):
        """medium: dict(Z, n, k_min, axis, lo, hi) or None (Sec. III E matter)."""
        if medium is None:
            self.L.or_set_medium(self.ctx, None)
            return
        m = Medium(int(medium["Z"]), float(medium["n"]), float(medium["k_min"]), int(medium.get("axis", 2)),
                   float(medium.get("lo", -1e300)), float(medium.get("hi", 1e300)))
        self.L.or_set_medium(self.ctx, C.byref(m))

    def medium_sigma(self, which, E):
        return self.L.or_medium_sigma(self.ctx, int(which), float(E))

    def medium_sample(self, which, E, r):
        return self.L.or_medium_sample(self.ctx, int(which), float(E), float(r))

    def table(self, which):
        n = C.c_uint64()
        p = self.L.or_table(self.ctx, int(which), C.byref(n))
        return np.ctypeslib.as_array(p, shape=(n.value,)).copy()


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return list(o)


def uniforms(seed, pid, step, ctr):
    o = np.zeros(2)
    lib().or_uniforms(int(seed), int(pid), int(step), int(ctr), _dp(o))
    return o


def besselk_scaled(x):
    o = np.zeros(3)
    lib().or_besselk_scaled(float(x), _dp(o))
    return o


def screening(g, e):
    o = np.zeros(4)
    lib().or_screening(float(g), float(e), _dp(o))
    return o


def coulomb_f(Z):
    return lib().or_coulomb_f(int(Z))


def brems_D(Z, E, y):
    return lib().or_brems_D(int(Z), float(E), float(y))


def pair_D(Z, k, x):
    return lib().or_pair_D(int(Z), float(k), float(x))


def scorer_gi_prime(y):
    return lib().or_scorer_gi_prime(float(y))


def field(f, x, y, z, t):
    E, B = np.zeros(3), np.zeros(3)
    lib().or_field(C.byref(f), float(x), float(y), float(z), float(t), _dp(E), _dp(B))
    return E, B


_KIND = {"none": FIELD_NONE, "uniform": FIELD_UNIFORM, "plane": FIELD_PLANE,
         "gauss": FIELD_GAUSS, "grid2d": FIELD_GRID2D}


def fields_from_spec(spec: dict, grid=None):
    """Field descriptor dict (as produced by ``workloads``) -> oracle Fields."""
    return make_fields(kind=_KIND[spec["kind"]], circular=int(spec.get("circular", 0)),
                       a0=float(spec.get("a0", 0.0)), phi0=float(spec.get("phi0", 0.0)),
                       length=float(spec.get("len", 1.0)), w0=float(spec.get("w0", 1.0)),
                       zf=float(spec.get("zf", 0.0)), E=spec.get("E", (0, 0, 0)),
                       B=spec.get("B", (0, 0, 0)), grid=grid)


class Sim:
    """One oracle simulation: e-, e+, photon arrays plus the id counter."""

    def __init__(self, orc: Oracle, wl: dict, cap_e=None, cap_p=None, cap_ph=None):
        self.o = orc
        ne, npos, nph = len(wl["e"]["id"]), len(wl["pos"]["id"]), len(wl["ph"]["id"])
        self.e = ParticleArrays(cap_e if cap_e is not None else max(4 * (ne + nph), 16)).load(wl["e"])
        self.pos = ParticleArrays(cap_p if cap_p is not None else max(4 * (ne + npos + nph), 16)).load(wl["pos"])
        self.ph = ParticleArrays(cap_ph if cap_ph is not None else max(8 * (ne + npos + nph), 16),
                                 photon=True).load(wl["ph"])
        self.fields = fields_from_spec(wl["field"], wl.get("grid"))
        self.dt = float(wl["dt"])
        self.t = float(wl.get("t0", 0.0))
        self.seed = int(wl["seed"])
        self.step_no = int(wl.get("step0", 0))
        orc.set_next_id(int(wl["next_id"]))
        orc.set_medium(wl.get("medium"))

    def run(self, nsteps, flags):
        tot = {}
        for _ in range(nsteps):
            s = self.o.step(self.e, self.pos, self.ph, self.fields, self.t, self.dt, self.seed,
                            self.step_no, flags)
            for k, v in s.items():
                tot[k] = tot.get(k, 0) + v
            self.t += self.dt
            self.step_no += 1
        return tot

    def decide(self, flags):
        """One step's decisions (Oracle.step_decide); the clock advances at commit."""
        return self.o.step_decide(self.e, self.pos, self.ph, self.fields, self.t, self.dt, self.seed,
                                  self.step_no, flags)

    def commit(self, bases=None):
        s = self.o.step_commit(self.e, self.pos, self.ph, bases)
        self.t += self.dt
        self.step_no += 1
        return s

    def load(self, st: dict):
        """Replace the particle arrays (e.g. reordered) and the id counter."""
        self.e.load(st["e"]); self.pos.load(st["pos"]); self.ph.load(st["ph"])
        self.o.set_next_id(int(st["next_id"]))

    def state(self):
        return {"e": self.e.view(), "pos": self.pos.view(), "ph": self.ph.view(),
                "next_id": self.o.next_id()}


# ---------------------------------------------------------------------------------
# Self-consistent 2D3V PIC around the step (Secs. II B, II C, II F): Yee solver and
# Esirkepov deposition of the oracle, driven in the paper's leapfrog order.
# ---------------------------------------------------------------------------------
class YeeGrid:
    """Double-precision Yee arrays [ny][nx] (E, B, J) with the oracle's solver."""

    NAMES = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz")

    def __init__(self, nx, ny, dx, dy, periodic=1, fields=None):
        self.a = {k: np.zeros((ny, nx)) for k in self.NAMES}
        if fields:
            for k, v in fields.items():
                self.a[k][...] = v
        self.g = Grid()
        for k in self.NAMES:
            setattr(self.g, k, _dp(self.a[k]))
        self.g.nx, self.g.ny, self.g.dx, self.g.dy, self.g.periodic = nx, ny, dx, dy, periodic
        self.L = lib()

    def advance_b(self, dt):
        self.L.or_fdtd_b(C.byref(self.g), float(dt))

    def advance_e(self, dt):
        self.L.or_fdtd_e(C.byref(self.g), float(dt))

    def charge(self, x, y, qw, x0=0.0, y0=0.0):
        rho = np.zeros((self.g.ny, self.g.nx))
        x, y, qw = map(_vec, (x, y, qw))
        self.L.or_charge_tsc(C.byref(self.g), float(x0), float(y0), _dp(x), _dp(y), _dp(qw), len(x), _dp(rho))
        return rho

    def div_e(self):
        a, g = self.a, self.g
        # div E at the nodes (i, j): Ex(i+1/2) - Ex(i-1/2), Ey(j+1/2) - Ey(j-1/2)
        ex, ey = a["Ex"], a["Ey"]
        if g.periodic:
            return (ex - np.roll(ex, 1, 1)) / g.dx + (ey - np.roll(ey, 1, 0)) / g.dy
        d = ex.copy() / g.dx
        d[:, 1:] -= ex[:, :-1] / g.dx
        d += ey / g.dy
        d[1:, :] -= ey[:-1, :] / g.dy
        return d


class PicSim(Sim):
    """The QED step inside the PIC loop of Fig. fig-loop, leapfrog of Sec. II F:
    E^n, B^{n-1/2} stored; B -> B^n by half a curl step; the step gathers (E^n, B^n),
    pushes, runs the QED processes and deposits J^{n+1/2} from x^n -> x^{n+1}; B -> B^{n+1/2}
    by the second half; E -> E^{n+1} with curl B^{n+1/2} - J^{n+1/2}.  The gather reads a
    float copy of the fields, as the grid is FP32 by specification."""

    def __init__(self, orc, wl, grid: YeeGrid, x0=0.0, y0=0.0, **caps):
        g = grid.g
        spec = {"Ex": np.zeros((g.ny, g.nx), np.float32), "dx": g.dx, "dy": g.dy, "x0": x0, "y0": y0,
                "periodic": g.periodic}
        for k in ("Ey", "Ez", "Bx", "By", "Bz"):
            spec[k] = np.zeros((g.ny, g.nx), np.float32)
        wl = dict(wl)
        wl["field"] = {"kind": "grid2d"}
        wl["grid"] = spec
        super().__init__(orc, wl, **caps)
        self.grid = grid
        f = self.fields
        for name, k in (("gJx", "Jx"), ("gJy", "Jy"), ("gJz", "Jz")):
            setattr(f, name, _dp(grid.a[k]))
        self._f32 = f._keep   # the float copies the gather reads (Ex..Bz)

    def _refresh(self):
        for arr, k in zip(self._f32, ("Ex", "Ey", "Ez", "Bx", "By", "Bz")):
            arr[...] = self.grid.a[k]

    def run(self, nsteps, flags):
        tot = {}
        for _ in range(nsteps):
            self.grid.advance_b(0.5 * self.dt)
            self._refresh()
            for k in ("Jx", "Jy", "Jz"):
                self.grid.a[k][...] = 0.0
            s = self.o.step(self.e, self.pos, self.ph, self.fields, self.t, self.dt, self.seed, self.step_no,
                            flags | F_DEPOSIT)
            for k, v in s.items():
                tot[k] = tot.get(k, 0) + v
            self.grid.advance_b(0.5 * self.dt)
            self.grid.advance_e(self.dt)
            self.t += self.dt
            self.step_no += 1
        return tot
