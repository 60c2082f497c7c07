"""CPU oracle of the PIC-DSMC time step -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It loads ``pd_oracle.c`` (plain C, built
here with gcc) through ctypes and shares nothing with the CUDA library except
the seeded inputs of :mod:`synthetic`.

Two builds of the same source: ``Oracle(cfg, fp64=True)`` keeps every particle
quantity in double (physics checks); ``fp64=False`` is the float mirror whose
operations follow the method's FP32 state step for step (bit-exact parity).
"""
import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "pd_oracle.c")


def compile_source(src, so, fp64, omp=False):
    """Compile the oracle source file `src` into the shared object `so` with
    the flags of the regular builds (omp: the build that runs on all host
    cores)."""
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", *(["-DOR_DOUBLE"] if fp64 else []), *(["-fopenmp", "-DOR_OMP"] if omp else []),
           "-o", so, src, "-lm"]
    subprocess.check_call(cmd)


BUILDS = (("oracle32", False, False), ("oracle64", True, False), ("oracle32_omp", False, True),
          ("oracle64_omp", True, True))


def build(force=False):
    """Compile the oracle builds with gcc (no fused multiply-add): double and
    float, each single-threaded and on all cores (OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    outs = {}
    for name, fp64, omp in BUILDS:
        so = os.path.join(_BUILD, f"lib{name}.so")
        if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
            tmp = so + f".tmp{os.getpid()}"
            compile_source(_SRC, tmp, fp64=fp64, omp=omp)
            os.replace(tmp, so)
        outs[name] = so
    return outs


class _Cfg(C.Structure):
    _fields_ = [
        ("geom", C.c_int32), ("nz", C.c_int32), ("nr", C.c_int32),
        ("dz", C.c_double), ("dr", C.c_double), ("depth", C.c_double), ("dt", C.c_double),
        ("heavy_subcycle", C.c_int32), ("weight", C.c_double),
        ("seed", C.c_uint32), ("run", C.c_uint32),
        ("field_mode", C.c_int32), ("inject_on", C.c_int32), ("di_on", C.c_int32),
        ("di_split_mode", C.c_int32), ("coll_dt_scale", C.c_double),
        ("V0", C.c_double), ("R_ohm", C.c_double), ("C_farad", C.c_double),
        ("beta", C.c_double), ("tip_radius", C.c_double), ("work_function", C.c_double),
        ("neutral_ratio", C.c_double), ("neutral_T", C.c_double),
        ("poisson_tol", C.c_double), ("capacity", C.c_int64), ("heavy_coll", C.c_int32),
        ("charge_max", C.c_int32), ("coulomb", C.c_int32), ("coulomb_lnl", C.c_double),
        ("sputter", C.c_int32), ("sputter_T", C.c_double),
    ]


_LIBS = {}
P = C.c_void_p
D = C.POINTER(C.c_double)


def _lib(fp64, omp=False):
    key = ("oracle64" if fp64 else "oracle32") + ("_omp" if omp else "")
    if key not in _LIBS:
        _LIBS[key] = bind(build()[key])
    return _LIBS[key]


def bind(so):
    """Load one build of the oracle from the shared object `so` and declare
    its entry points (the tests also bind builds they compile themselves)."""
    L = C.CDLL(so)
    L.or_create.restype = P
    L.or_create.argtypes = [C.POINTER(_Cfg)]
    L.or_destroy.argtypes = [P]
    L.or_set_xs.argtypes = [P, C.c_int, D, D, C.c_int, C.c_double]
    L.or_set_yield.argtypes = [P, D, D, C.c_int]
    L.or_load.restype = C.c_int64
    L.or_load.argtypes = [P, C.c_int64, P, P, P, D, D, D, D, D]
    L.or_set_field.argtypes = [P, D, D]
    L.or_step.argtypes = [P, C.c_int]
    L.or_prime.argtypes = [P]
    L.or_count.restype = C.c_int64
    L.or_count.argtypes = [P]
    L.or_get_particles.argtypes = [P, P, P, P, P, D, D, D, D, D]
    L.or_get_rho.argtypes = [P, P, P]
    L.or_get_phi.argtypes = [P, D]
    L.or_get_field.argtypes = [P, D, D]
    L.or_get_counters.argtypes = [P, P]
    L.or_get_scalars.argtypes = [P, D]
    L.or_density_map.argtypes = [P, C.c_int, D]
    L.or_energy_spectrum.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_int, P]
    L.or_poisson_solve.argtypes = [P, D, C.c_double, C.c_double, D]
    L.or_efield.argtypes = [P, D, D, D]
    L.or_node_volume.restype = C.c_double
    L.or_node_volume.argtypes = [P, C.c_int, C.c_int]
    L.or_cell_volume.restype = C.c_double
    L.or_cell_volume.argtypes = [P, C.c_int]
    L.or_xs_lookup_d.restype = C.c_double
    L.or_xs_lookup_d.argtypes = [P, C.c_int, C.c_double]
    L.or_fn_current.restype = C.c_double
    L.or_fn_current.argtypes = [C.c_double, C.c_double]
    L.or_philox.argtypes = [P, P, P]
    L.or_event_kinematics.argtypes = [P, C.c_int, C.c_uint32, C.c_uint32, C.c_uint32, D, D, D, P]
    L.or_rectangle_split.argtypes = [P, C.c_uint32, C.c_uint32, C.c_uint32, D, D, D]
    L.or_deposit_weights.argtypes = [C.c_double, C.c_double, P, P]
    L.or_coulomb_kinematics.argtypes = [P, C.c_uint32, C.c_uint32, C.c_uint32, D, D, C.c_double, C.c_double,
                                        C.c_double]
    L.or_perm_index.restype = C.c_uint32
    L.or_perm_index.argtypes = [C.c_uint32, C.c_uint32, P]
    return L


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _dptr(a):
    return a.ctypes.data_as(D)


COUNTER_NAMES = (["ev_el", "ev_exc", "ev_si", "ev_di", "ev_sw", "nulls", "consumed", "thr_rej",
                  "ratio_viol", "iso_fallback", "cand_total", "emitted_e", "emitted_cu"]
                 + [f"abs_{e}_{s}" for e in ("cathode", "anode", "wall")
                    for s in ("e", "Cu", "Cu+", "Cu2+SW", "Cu2+DI", "Cu3+", "Cu4+")]
                 + ["ev_cx", "ev_nn", "ev_s3", "ev_s4", "coul_ee", "coul_ei", "sput_cathode", "sput_anode",
                    "coul_ii"])
SCALAR_NAMES = ["t", "V", "I_gap", "gamma", "Qbar", "erosion", "mass", "charge", "sgmax0",
                "sgmax1", "poisson_relres", "poisson_iters", "E_abs_cathode", "E_abs_anode",
                "E_abs_wall"]


def philox4x32_10(ctr, key):
    L = _lib(False)
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    L.or_philox(_ptr(c), _ptr(k), _ptr(o))
    return o


def fn_current(F, work):
    return _lib(False).or_fn_current(float(F), float(work))


class Oracle:
    """One CPU simulation.  `cfg` is a :func:`synthetic.base_config` dict."""

    def __init__(self, cfg, fp64=True, field_mode=None, lib=None, omp=False):
        self.L = _lib(fp64, omp) if lib is None else lib
        self.fp64 = fp64
        self.cfg = dict(cfg)
        c = _Cfg()
        c.geom = 0 if cfg["geometry"] == "rz" else 1
        c.nz, c.nr = cfg["nz"], cfg["nr"]
        c.dz, c.dr, c.depth, c.dt = cfg["dz"], cfg["dr"], cfg.get("depth", 1.0), cfg["dt"]
        c.heavy_subcycle = cfg["heavy_subcycle"]
        c.weight = cfg["weight"]
        c.seed, c.run = cfg["seed"], cfg.get("run", 0)
        c.field_mode = cfg["field_on"] if field_mode is None else field_mode
        c.inject_on, c.di_on = cfg["inject_on"], cfg["di_on"]
        c.di_split_mode = cfg.get("di_split_mode", 0)
        c.coll_dt_scale = cfg.get("coll_dt_scale", 1.0)
        c.V0, c.R_ohm, c.C_farad = cfg["V0"], cfg["R_ohm"], cfg["C_farad"]
        c.beta, c.tip_radius, c.work_function = cfg["beta"], cfg["tip_radius"], cfg["work_function"]
        c.neutral_ratio, c.neutral_T = cfg["neutral_ratio"], cfg["neutral_T"]
        c.poisson_tol = cfg.get("oracle_poisson_tol", 1e-11)
        c.capacity = cfg["capacity"]
        c.heavy_coll = cfg.get("heavy_coll", 0)
        c.charge_max = cfg.get("charge_max", 2)
        c.coulomb = cfg.get("coulomb", 0)
        c.coulomb_lnl = cfg.get("coulomb_lnl", 10.0)
        c.sputter = cfg.get("sputter", 0)
        c.sputter_T = cfg.get("sputter_T", 23209.0)
        self._c = c
        self.h = self.L.or_create(C.byref(c))
        rz = c.geom == 0
        self.nzn = cfg["nz"] + 1 if rz else cfg["nz"]
        self.nrn = cfg["nr"] + 1 if rz else cfg["nr"]

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.or_destroy(h)
            self.h = None

    def set_cross_sections(self, xs):
        for ch, (E, s, th) in xs.items():
            E = np.ascontiguousarray(E, np.float64)
            s = np.ascontiguousarray(s, np.float64)
            self.L.or_set_xs(self.h, int(ch), _dptr(E), _dptr(s), len(E), float(th))

    def set_sputter_yield(self, E, Y):
        """Sputtering yield (atoms per ion) against impact energy (eV)."""
        E = np.ascontiguousarray(E, np.float64)
        Y = np.ascontiguousarray(Y, np.float64)
        if self.L.or_set_yield(self.h, _dptr(E), _dptr(Y), len(E)):
            raise ValueError("yield table needs at least two points")

    def load(self, parts):
        n = len(parts["species"])
        sp = np.ascontiguousarray(parts["species"], np.uint8)
        iz = np.ascontiguousarray(parts["iz"], np.int32)
        ir = np.ascontiguousarray(parts["ir"], np.int32)
        arr = [np.ascontiguousarray(parts[k], np.float64) for k in ("pz", "pr", "vz", "vr", "vt")]
        r = self.L.or_load(self.h, n, _ptr(sp), _ptr(iz), _ptr(ir), *[_dptr(a) for a in arr])
        if r == -2:
            raise ValueError("species code above the configured highest charge")
        if r < 0:
            raise RuntimeError("oracle capacity exceeded")

    def set_field(self, Ez, Er):
        Ez = np.ascontiguousarray(Ez, np.float64).ravel()
        Er = np.ascontiguousarray(Er, np.float64).ravel()
        self.L.or_set_field(self.h, _dptr(Ez), _dptr(Er))

    def prime(self):
        self.L.or_prime(self.h)

    def step(self, n=1):
        r = self.L.or_step(self.h, int(n))
        if r:
            raise RuntimeError(f"oracle step failed ({r})")

    def count(self):
        return int(self.L.or_count(self.h))

    def particles(self):
        n = self.count()
        out = dict(id=np.zeros(n, np.uint32), species=np.zeros(n, np.uint8),
                   iz=np.zeros(n, np.int32), ir=np.zeros(n, np.int32))
        for k in ("pz", "pr", "vz", "vr", "vt"):
            out[k] = np.zeros(n, np.float64)
        self.L.or_get_particles(self.h, _ptr(out["id"]), _ptr(out["species"]), _ptr(out["iz"]),
                                _ptr(out["ir"]), *[_dptr(out[k]) for k in ("pz", "pr", "vz", "vr", "vt")])
        return out

    def rho(self):
        nn = self.nzn * self.nrn
        a = np.zeros(nn, np.int64)
        b = np.zeros(nn, np.int64)
        self.L.or_get_rho(self.h, _ptr(a), _ptr(b))
        return a.reshape(self.nzn, self.nrn), b.reshape(self.nzn, self.nrn)

    def phi(self):
        a = np.zeros(self.nzn * self.nrn)
        self.L.or_get_phi(self.h, _dptr(a))
        return a.reshape(self.nzn, self.nrn)

    def field(self):
        a = np.zeros(self.nzn * self.nrn)
        b = np.zeros(self.nzn * self.nrn)
        self.L.or_get_field(self.h, _dptr(a), _dptr(b))
        return a.reshape(self.nzn, self.nrn), b.reshape(self.nzn, self.nrn)

    def counters(self):
        a = np.zeros(len(COUNTER_NAMES), np.uint64)
        self.L.or_get_counters(self.h, _ptr(a))
        return dict(zip(COUNTER_NAMES, (int(x) for x in a)))

    def scalars(self):
        a = np.zeros(len(SCALAR_NAMES))
        self.L.or_get_scalars(self.h, _dptr(a))
        return dict(zip(SCALAR_NAMES, (float(x) for x in a)))

    def density_map(self, species):
        a = np.zeros(self.nzn * self.nrn)
        self.L.or_density_map(self.h, int(species), _dptr(a))
        return a.reshape(self.nzn, self.nrn)

    def energy_spectrum(self, species, lo=0.0, hi=500.0, nbins=100):
        a = np.zeros(nbins, np.uint64)
        self.L.or_energy_spectrum(self.h, int(species), lo, hi, nbins, _ptr(a))
        return a

    def poisson(self, rho, V, tol=1e-12, phi0=None):
        rho = np.ascontiguousarray(rho, np.float64).ravel()
        phi = np.zeros(self.nzn * self.nrn) if phi0 is None else np.ascontiguousarray(phi0, np.float64).ravel().copy()
        it = self.L.or_poisson_solve(self.h, _dptr(rho), float(V), float(tol), _dptr(phi))
        return phi.reshape(self.nzn, self.nrn), it

    def efield(self, phi):
        phi = np.ascontiguousarray(phi, np.float64).ravel()
        a = np.zeros_like(phi)
        b = np.zeros_like(phi)
        self.L.or_efield(self.h, _dptr(phi), _dptr(a), _dptr(b))
        return a.reshape(self.nzn, self.nrn), b.reshape(self.nzn, self.nrn)

    def node_volume(self, i, j):
        return self.L.or_node_volume(self.h, i, j)

    def cell_volume(self, j):
        return self.L.or_cell_volume(self.h, j)

    def xs_lookup(self, ch, eps):
        return self.L.or_xs_lookup_d(self.h, ch, float(eps))

    def event(self, ch, ve, vt, subject=0, step=0, sid=0):
        ve = np.array(ve, np.float64)
        vt = np.array(vt, np.float64)
        en = np.zeros(6)
        ns = C.c_int(0)
        r = self.L.or_event_kinematics(self.h, ch, subject, step, sid, _dptr(ve), _dptr(vt),
                                       _dptr(en), C.byref(ns))
        if r < 0:
            return None
        return ve, vt, [en[0:3].copy(), en[3:6].copy()][: ns.value]

    def coulomb(self, va, vb, Kn, fa, fb, subject=0, step=0, sid=0):
        """One Coulomb pair collision (binary collision model); None if the
        relative velocity is zero."""
        va = np.array(va, np.float64)
        vb = np.array(vb, np.float64)
        r = self.L.or_coulomb_kinematics(self.h, subject, step, sid, _dptr(va), _dptr(vb), float(Kn), float(fa),
                                         float(fb))
        return (va, vb) if r else None

    def rectangle_split(self, v, subject=0, step=0, sid=0):
        v = np.array(v, np.float64)
        a = np.zeros(3)
        b = np.zeros(3)
        self.L.or_rectangle_split(self.h, subject, step, sid, _dptr(v), _dptr(a), _dptr(b))
        return a, b


def perm_index(x, n, key):
    """Element x of the keyed pseudo-random permutation of [0, n)."""
    k = np.asarray(key, np.uint32)
    return int(_lib(False).or_perm_index(int(x), int(n), _ptr(k)))


def deposit_weights(pz, pr, fp64=False):
    wz = C.c_uint32(0)
    wr = C.c_uint32(0)
    _lib(fp64).or_deposit_weights(float(pz), float(pr), C.byref(wz), C.byref(wr))
    return wz.value, wr.value
