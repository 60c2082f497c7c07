"""Python binding of libpd.so (include/pd.h): argument marshalling only.

Every step of the particle pipeline runs in the library's CUDA kernels; this
module only fills the C structs, passes torch tensors' device pointers and
CUDA streams, and copies host arrays in and out.  Importing it loads the
compiled library and fails loudly if it is missing: there is no fallback.

The functions keep the C names (pd_create, pd_step, ...).  ``Simulation`` is
a small convenience holder of a workspace tensor and a pd_sim handle.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = ["PdConfig", "PdScalars", "Simulation", "PdError", "load_library", "config_from_dict",
           "pd_config_default", "pd_workspace_size", "pd_create", "pd_set_cross_section", "pd_set_sputter_yield",
           "pd_load_particles", "pd_load_particles_device", "pd_set_field", "pd_inject_cathode",
           "pd_step", "pd_synchronize", "pd_get_scalars", "pd_get_counters", "pd_particle_slots", "pd_get_sort_stats", "pd_get_bins", "pd_spectrum_static_max_bins",
           "pd_get_particles", "pd_get_rho", "pd_get_phi", "pd_get_field", "pd_get_density_map",
           "pd_get_energy_spectrum", "pd_profile_enable", "pd_profile_read", "pd_kernel_name",
           "pd_last_error", "pd_destroy", "pd_energy_spectrum_static", "Ensemble", "pd_ensemble_workspace_size",
           "pd_ensemble_create", "pd_ensemble_step", "pd_ensemble_get_scalars", "pd_run_count", "pd_run_layout",
           "pd_get_run_counters", "pd_get_run_density_map", "pd_get_run_energy_spectrum", "pd_load_particles_run",
           "pd_load_particles_device_run", "pd_set_graph_mode", "PdTuning", "pd_get_tuning",
           "pd_set_tuning", "pd_autotune", "pd_save", "pd_load", "pd_get_rho_phi", "Net", "PD_NET_NPARAMS", "pd_net_workspace_size",
           "pd_net_create", "pd_net_destroy", "pd_net_set_params", "pd_net_get_params", "pd_net_forward",
           "pd_net_loss_grad", "pd_net_loss_grad_rz", "pd_net_adam", "pd_warmstart_pairs", "pd_set_warm_start", "WARM_MODES",
           "COUNTER_NAMES", "KERNEL_NAMES", "EXPORTED"]

PD_NCOUNTERS = 43
PD_NKERNELS = 13
GEOM = {"rz": 0, "xy_periodic": 1}
COUNTER_NAMES = (["ev_el", "ev_exc", "ev_si", "ev_di", "ev_sw", "nulls", "consumed", "thr_rej",
                  "ratio_viol", "iso_fallback", "cand_total", "emitted_e", "emitted_cu"]
                 + [f"abs_{e}_{s}" for e in ("cathode", "anode", "wall")
                    for s in ("e", "Cu", "Cu+", "Cu2+SW", "Cu2+DI", "Cu3+", "Cu4+")]
                 + ["ev_cx", "ev_nn", "ev_s3", "ev_s4", "coul_ee", "coul_ei", "sput_cathode", "sput_anode",
                    "coul_ii"])
STATUS = {0: "PD_OK", 1: "PD_ERR_ARG", 2: "PD_ERR_CAPACITY", 3: "PD_ERR_CUDA", 4: "PD_ERR_TIMEOUT",
          5: "PD_ERR_NONFINITE", 6: "PD_ERR_STATE"}


class PdConfig(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("version", C.c_uint32), ("geometry", C.c_int32),
        ("nz", C.c_int32), ("nr", C.c_int32), ("dz", C.c_double), ("dr", C.c_double),
        ("depth", C.c_double), ("dt", C.c_double), ("heavy_subcycle", C.c_int32),
        ("weight", C.c_double), ("seed", C.c_uint32), ("run", C.c_uint32),
        ("field_mode", C.c_int32), ("inject_on", C.c_int32), ("di_on", C.c_int32),
        ("di_split_mode", C.c_int32), ("coll_dt_scale", C.c_double), ("V0", C.c_double),
        ("R_ohm", C.c_double), ("C_farad", C.c_double), ("beta", C.c_double),
        ("tip_radius", C.c_double), ("work_function", C.c_double), ("neutral_ratio", C.c_double),
        ("neutral_T", C.c_double), ("poisson_tol", C.c_double), ("poisson_max_cycles", C.c_int32),
        ("heavy_coll", C.c_int32), ("charge_max", C.c_int32), ("coulomb", C.c_int32),
        ("capacity", C.c_int64), ("coulomb_lnl", C.c_double), ("sputter", C.c_int32), ("reserved1", C.c_int32),
        ("sputter_T", C.c_double),
    ]


class PdScalars(C.Structure):
    _fields_ = [
        ("t", C.c_double), ("V", C.c_double), ("I_gap", C.c_double), ("gamma", C.c_double),
        ("Qbar", C.c_double), ("erosion", C.c_double), ("mass", C.c_double), ("charge", C.c_double),
        ("sgmax", C.c_double * 2), ("poisson_relres", C.c_double), ("poisson_cycles", C.c_double),
        ("poisson_relres_max", C.c_double), ("poisson_relres0", C.c_double),
        ("absorbed_energy", C.c_double * 3), ("n_particles", C.c_int64), ("count", C.c_int64 * 7),
        ("step", C.c_int64),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


class PdTuning(C.Structure):
    _fields_ = [
        ("push_blocks_per_sm", C.c_int32), ("bincount_blocks_per_sm", C.c_int32),
        ("scatter_blocks_per_sm", C.c_int32), ("ncand_blocks_per_sm", C.c_int32),
        ("collide_blocks_per_sm", C.c_int32), ("mg_threads", C.c_int32), ("mg_max_blocks", C.c_int32),
    ]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class PdError(RuntimeError):
    pass


_L = None
P = C.c_void_p
Dp = C.POINTER(C.c_double)

_SIGS = {
    "pd_config_default": (C.c_int, [C.POINTER(PdConfig)]),
    "pd_workspace_size": (C.c_int, [C.POINTER(PdConfig), C.POINTER(C.c_size_t)]),
    "pd_create": (C.c_int, [C.POINTER(PdConfig), P, C.c_size_t, P, C.POINTER(P)]),
    "pd_set_cross_section": (C.c_int, [P, C.c_int, Dp, Dp, C.c_int, C.c_double]),
    "pd_set_sputter_yield": (C.c_int, [P, Dp, Dp, C.c_int]),
    "pd_load_particles": (C.c_int, [P, C.c_int64, P, P, P, P, P, P, P, P]),
    "pd_load_particles_device": (C.c_int, [P, C.c_int64, P, P, P, P, P, P, P, P]),
    "pd_set_field": (C.c_int, [P, Dp, Dp]),
    "pd_inject_cathode": (C.c_int, [P, C.c_int]),
    "pd_step": (C.c_int, [P, C.c_int64]),
    "pd_synchronize": (C.c_int, [P]),
    "pd_get_scalars": (C.c_int, [P, C.POINTER(PdScalars)]),
    "pd_get_counters": (C.c_int, [P, P]),
    "pd_particle_slots": (C.c_int, [P, C.POINTER(C.c_int64)]),
    "pd_get_sort_stats": (C.c_int, [P, P]),
    "pd_spectrum_static_max_bins": (C.c_int, []),
    "pd_get_bins": (C.c_int, [P, P, P, C.POINTER(C.c_int64)]),
    "pd_get_particles": (C.c_int, [P, P, P, P, P, P, P, P, P, P, P]),
    "pd_ensemble_workspace_size": (C.c_int, [C.POINTER(PdConfig), C.c_int, C.POINTER(C.c_size_t)]),
    "pd_ensemble_create": (C.c_int, [C.POINTER(PdConfig), C.c_int, P, C.c_size_t, P, C.POINTER(P)]),
    "pd_ensemble_step": (C.c_int, [P, C.c_int64]),
    "pd_ensemble_get_scalars": (C.c_int, [P, C.c_int, C.POINTER(PdScalars)]),
    "pd_run_count": (C.c_int, [P, C.POINTER(C.c_int)]),
    "pd_run_layout": (C.c_int, [P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "pd_get_run_counters": (C.c_int, [P, C.c_int, P]),
    "pd_get_run_density_map": (C.c_int, [P, C.c_int, C.c_int, Dp]),
    "pd_get_run_energy_spectrum": (C.c_int, [P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, P]),
    "pd_load_particles_run": (C.c_int, [P, C.c_int, C.c_int64, P, P, P, P, P, P, P, P]),
    "pd_load_particles_device_run": (C.c_int, [P, C.c_int, C.c_int64, P, P, P, P, P, P, P, P]),
    "pd_set_graph_mode": (C.c_int, [P, C.c_int, C.c_int]),
    "pd_get_tuning": (C.c_int, [P, C.POINTER(PdTuning)]),
    "pd_set_tuning": (C.c_int, [P, C.POINTER(PdTuning)]),
    "pd_autotune": (C.c_int, [P, C.c_int, C.POINTER(PdTuning)]),
    "pd_save": (C.c_int, [P, C.c_char_p]),
    "pd_load": (C.c_int, [P, C.c_char_p]),
    "pd_get_rho_phi": (C.c_int, [P, Dp, Dp]),
    "pd_net_workspace_size": (C.c_int, [C.c_int64, C.POINTER(C.c_size_t)]),
    "pd_net_create": (C.c_int, [C.c_int64, P, C.c_size_t, P, C.POINTER(P)]),
    "pd_net_destroy": (None, [P]),
    "pd_net_set_params": (C.c_int, [P, P]),
    "pd_net_get_params": (C.c_int, [P, P]),
    "pd_net_forward": (C.c_int, [P, P, C.c_int, C.c_int, C.c_int, P]),
    "pd_net_loss_grad": (C.c_int, [P, P, P, C.c_int, C.c_int, C.c_int, Dp, P]),
    "pd_net_loss_grad_rz": (C.c_int, [P, P, C.c_int, C.c_int, C.c_int, Dp, P]),
    "pd_net_adam": (C.c_int, [P, C.c_float, C.c_float, C.c_float, C.c_float]),
    "pd_warmstart_pairs": (C.c_int, [P, C.c_int, P, P]),
    "pd_set_warm_start": (C.c_int, [P, C.c_int, P]),
    "pd_get_rho": (C.c_int, [P, P, P]),
    "pd_get_phi": (C.c_int, [P, Dp]),
    "pd_get_field": (C.c_int, [P, Dp, Dp]),
    "pd_get_density_map": (C.c_int, [P, C.c_int, Dp]),
    "pd_get_energy_spectrum": (C.c_int, [P, C.c_int, C.c_double, C.c_double, C.c_int, P]),
    "pd_profile_enable": (C.c_int, [P, C.c_int]),
    "pd_profile_read": (C.c_int, [P, Dp, P]),
    "pd_kernel_name": (C.c_char_p, [C.c_int]),
    "pd_last_error": (C.c_char_p, [P]),
    "pd_destroy": (None, [P]),
    "pd_energy_spectrum_static": (C.c_int, [P, P, P, P, C.c_int64, C.c_int, C.c_double, C.c_double, C.c_int,
                                            P, P]),
}
EXPORTED = tuple(_SIGS)


def load_library(path=None, build_if_missing=True):
    """Load libpd.so (building it with nvcc if it is absent or stale)."""
    global _L
    if _L is not None:
        return _L
    if path is None:
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
    if not os.path.exists(path):
        raise PdError(f"CUDA library {path} is missing; build it with paper_2109_00214_gb300/build.py")
    L = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _L = L
    return L


def _lib():
    return _L if _L is not None else load_library()


def _ptr(a):
    return C.c_void_p(a.ctypes.data)


def _dp(a):
    return a.ctypes.data_as(Dp)


def _check(h, r, what):
    if r != 0:
        msg = _lib().pd_last_error(h) if h else b""
        raise PdError(f"{what}: {STATUS.get(r, r)}: {msg.decode() if msg else ''}")


def config_from_dict(d):
    c = PdConfig()
    _check(None, _lib().pd_config_default(C.byref(c)), "pd_config_default")
    c.geometry = GEOM[d["geometry"]]
    c.nz, c.nr = d["nz"], d["nr"]
    c.dz, c.dr, c.depth, c.dt = d["dz"], d["dr"], d.get("depth", 1.0), d["dt"]
    c.heavy_subcycle = d["heavy_subcycle"]
    c.weight = d["weight"]
    c.seed, c.run = d["seed"], d.get("run", 0)
    c.field_mode = d["field_on"]
    c.inject_on, c.di_on = d["inject_on"], d["di_on"]
    c.di_split_mode = d.get("di_split_mode", 0)
    c.coll_dt_scale = d.get("coll_dt_scale", 1.0)
    c.V0, c.R_ohm, c.C_farad = d["V0"], d["R_ohm"], d["C_farad"]
    c.beta, c.tip_radius, c.work_function = d["beta"], d["tip_radius"], d["work_function"]
    c.neutral_ratio, c.neutral_T = d["neutral_ratio"], d["neutral_T"]
    c.poisson_tol = d.get("poisson_tol", 1e-8)
    c.poisson_max_cycles = d.get("poisson_max_cycles", 60)
    c.heavy_coll = d.get("heavy_coll", 0)
    c.charge_max = d.get("charge_max", 2)
    c.coulomb = d.get("coulomb", 0)
    c.coulomb_lnl = d.get("coulomb_lnl", 10.0)
    c.sputter = d.get("sputter", 0)
    c.sputter_T = d.get("sputter_T", 23209.0)
    c.capacity = d["capacity"]
    return c


# ---- thin wrappers with the C names --------------------------------------
def pd_config_default():
    c = PdConfig()
    _check(None, _lib().pd_config_default(C.byref(c)), "pd_config_default")
    return c


def pd_workspace_size(cfg):
    n = C.c_size_t(0)
    _check(None, _lib().pd_workspace_size(C.byref(cfg), C.byref(n)), "pd_workspace_size")
    return n.value


def pd_create(cfg, workspace_ptr, nbytes, stream_ptr):
    h = P()
    _check(None, _lib().pd_create(C.byref(cfg), P(workspace_ptr), nbytes, P(stream_ptr), C.byref(h)),
           "pd_create")
    return h


def pd_set_sputter_yield(h, E, Y):
    E = np.ascontiguousarray(E, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    _check(h, _lib().pd_set_sputter_yield(h, _dp(E), _dp(Y), len(E)), "pd_set_sputter_yield")


def pd_set_cross_section(h, ch, E, sig, threshold):
    E = np.ascontiguousarray(E, np.float64)
    sig = np.ascontiguousarray(sig, np.float64)
    _check(h, _lib().pd_set_cross_section(h, int(ch), _dp(E), _dp(sig), len(E), float(threshold)),
           "pd_set_cross_section")


def pd_load_particles(h, parts):
    n = len(parts["species"])
    a = [np.ascontiguousarray(parts["species"], np.uint8), np.ascontiguousarray(parts["iz"], np.int32),
         np.ascontiguousarray(parts["ir"], np.int32)]
    a += [np.ascontiguousarray(parts[k], np.float32) for k in ("pz", "pr", "vz", "vr", "vt")]
    _check(h, _lib().pd_load_particles(h, n, *[_ptr(x) for x in a]), "pd_load_particles")


def pd_load_particles_ptrs(h, n, ptrs):
    """Host pointers (int; pinned memory loads fastest) of species u8, iz i32,
    ir i32, pz, pr, vz, vr, vt f32."""
    _check(h, _lib().pd_load_particles(h, int(n), *[P(p) for p in ptrs]), "pd_load_particles")


def pd_load_particles_run_ptrs(h, run, n, ptrs):
    """As pd_load_particles_ptrs, into one run of an ensemble."""
    _check(h, _lib().pd_load_particles_run(h, int(run), int(n), *[P(p) for p in ptrs]), "pd_load_particles_run")


def pd_load_particles_device(h, n, ptrs):
    """ptrs: device pointers (int) of species u8, iz i32, ir i32, pz, pr, vz, vr, vt f32."""
    _check(h, _lib().pd_load_particles_device(h, int(n), *[P(p) for p in ptrs]), "pd_load_particles_device")


def pd_set_field(h, Ez, Er):
    Ez = np.ascontiguousarray(Ez, np.float64).ravel()
    Er = np.ascontiguousarray(Er, np.float64).ravel()
    _check(h, _lib().pd_set_field(h, _dp(Ez), _dp(Er)), "pd_set_field")


def pd_inject_cathode(h, enable):
    _check(h, _lib().pd_inject_cathode(h, int(enable)), "pd_inject_cathode")


def pd_step(h, n):
    _check(h, _lib().pd_step(h, int(n)), "pd_step")


def pd_synchronize(h):
    _check(h, _lib().pd_synchronize(h), "pd_synchronize")


def pd_get_scalars(h):
    s = PdScalars()
    _check(h, _lib().pd_get_scalars(h, C.byref(s)), "pd_get_scalars")
    return s.as_dict()


def pd_get_counters(h):
    a = np.zeros(PD_NCOUNTERS, np.uint64)
    _check(h, _lib().pd_get_counters(h, _ptr(a)), "pd_get_counters")
    return dict(zip(COUNTER_NAMES, (int(x) for x in a)))


class PdSortStats(C.Structure):
    _fields_ = [("relayouts", C.c_uint64), ("bin_slots", C.c_uint64), ("live", C.c_uint64),
                ("steps_since", C.c_uint64), ("faults", C.c_uint64)]


def pd_get_sort_stats(h):
    st = PdSortStats()
    _check(h, _lib().pd_get_sort_stats(h, C.byref(st)), "pd_get_sort_stats")
    return {name: int(getattr(st, name)) for name, _ in st._fields_}


def pd_get_bins(h):
    """(start, count) of the sort's bins: start has nbins + 1 entries (the
    last is the first slot of the tail)."""
    nb = C.c_int64(0)
    _check(h, _lib().pd_get_bins(h, None, None, C.byref(nb)), "pd_get_bins")
    start = np.zeros(nb.value + 1, np.uint32)
    count = np.zeros(nb.value, np.uint32)
    _check(h, _lib().pd_get_bins(h, _ptr(start), _ptr(count), C.byref(nb)), "pd_get_bins")
    return start, count


def pd_particle_slots(h):
    n = C.c_int64(0)
    _check(h, _lib().pd_particle_slots(h, C.byref(n)), "pd_particle_slots")
    return n.value


def pd_get_particles(h, live_only=True):
    n = pd_particle_slots(h)
    out = dict(id=np.zeros(n, np.uint32), run=np.zeros(n, np.int32), species=np.zeros(n, np.uint8),
               iz=np.zeros(n, np.int32), ir=np.zeros(n, np.int32))
    for k in ("pz", "pr", "vz", "vr", "vt"):
        out[k] = np.zeros(n, np.float32)
    keys = ("id", "run", "species", "iz", "ir", "pz", "pr", "vz", "vr", "vt")
    _check(h, _lib().pd_get_particles(h, *[_ptr(out[k]) for k in keys]), "pd_get_particles")
    if live_only:
        m = out["species"] != 255
        out = {k: v[m] for k, v in out.items()}
    return out


def pd_ensemble_workspace_size(cfgs):
    arr = (PdConfig * len(cfgs))(*cfgs)
    n = C.c_size_t(0)
    _check(None, _lib().pd_ensemble_workspace_size(arr, len(cfgs), C.byref(n)), "pd_ensemble_workspace_size")
    return n.value


def pd_ensemble_create(cfgs, workspace_ptr, nbytes, stream_ptr):
    arr = (PdConfig * len(cfgs))(*cfgs)
    h = P()
    _check(None, _lib().pd_ensemble_create(arr, len(cfgs), P(workspace_ptr), nbytes, P(stream_ptr), C.byref(h)),
           "pd_ensemble_create")
    return h


def pd_ensemble_step(h, n):
    _check(h, _lib().pd_ensemble_step(h, int(n)), "pd_ensemble_step")


def pd_ensemble_get_scalars(h, run):
    s = PdScalars()
    _check(h, _lib().pd_ensemble_get_scalars(h, int(run), C.byref(s)), "pd_ensemble_get_scalars")
    return s.as_dict()


def pd_run_count(h):
    n = C.c_int(0)
    _check(h, _lib().pd_run_count(h, C.byref(n)), "pd_run_count")
    return n.value


def pd_run_layout(h, run):
    a = C.c_int64(0)
    b = C.c_int64(0)
    _check(h, _lib().pd_run_layout(h, int(run), C.byref(a), C.byref(b)), "pd_run_layout")
    return a.value, b.value


def pd_get_run_counters(h, run):
    a = np.zeros(PD_NCOUNTERS, np.uint64)
    _check(h, _lib().pd_get_run_counters(h, int(run), _ptr(a)), "pd_get_run_counters")
    return dict(zip(COUNTER_NAMES, (int(x) for x in a)))


def pd_get_run_density_map(h, run, species, nodes):
    a = np.zeros(nodes)
    _check(h, _lib().pd_get_run_density_map(h, int(run), int(species), _dp(a)), "pd_get_run_density_map")
    return a


def pd_get_run_energy_spectrum(h, run, species, lo, hi, nbins):
    a = np.zeros(nbins, np.uint64)
    _check(h, _lib().pd_get_run_energy_spectrum(h, int(run), int(species), float(lo), float(hi), int(nbins),
                                                 _ptr(a)), "pd_get_run_energy_spectrum")
    return a


def pd_load_particles_run(h, run, parts):
    n = len(parts["species"])
    a = [np.ascontiguousarray(parts["species"], np.uint8), np.ascontiguousarray(parts["iz"], np.int32),
         np.ascontiguousarray(parts["ir"], np.int32)]
    a += [np.ascontiguousarray(parts[k], np.float32) for k in ("pz", "pr", "vz", "vr", "vt")]
    _check(h, _lib().pd_load_particles_run(h, int(run), n, *[_ptr(x) for x in a]), "pd_load_particles_run")


def pd_load_particles_device_run(h, run, n, ptrs):
    _check(h, _lib().pd_load_particles_device_run(h, int(run), int(n), *[P(p) for p in ptrs]),
           "pd_load_particles_device_run")


def pd_set_graph_mode(h, enable, poisson_cycles=4):
    _check(h, _lib().pd_set_graph_mode(h, int(enable), int(poisson_cycles)), "pd_set_graph_mode")


def pd_get_tuning(h):
    t = PdTuning()
    _check(h, _lib().pd_get_tuning(h, C.byref(t)), "pd_get_tuning")
    return t.as_dict()


def pd_set_tuning(h, **kw):
    """Change some launch shapes (keys of PdTuning); the others keep their values."""
    t = PdTuning()
    _check(h, _lib().pd_get_tuning(h, C.byref(t)), "pd_get_tuning")
    for k, v in kw.items():
        if k not in t.as_dict():
            raise KeyError(k)
        setattr(t, k, int(v))
    _check(h, _lib().pd_set_tuning(h, C.byref(t)), "pd_set_tuning")


def pd_autotune(h, steps_per_trial=2):
    t = PdTuning()
    _check(h, _lib().pd_autotune(h, int(steps_per_trial), C.byref(t)), "pd_autotune")
    return t.as_dict()


def pd_save(h, path):
    _check(h, _lib().pd_save(h, os.fsencode(path)), "pd_save")


def pd_load(h, path):
    _check(h, _lib().pd_load(h, os.fsencode(path)), "pd_load")


def pd_get_rho_phi(h, nodes):
    rho = np.zeros(nodes)
    phi = np.zeros(nodes)
    _check(h, _lib().pd_get_rho_phi(h, _dp(rho), _dp(phi)), "pd_get_rho_phi")
    return rho, phi


PD_NET_NPARAMS = 37601
WARM_MODES = {"previous": 0, "cold": 1, "learned": 2, "learned_delta": 3, "extrapolate": 4, "learned_extrap": 5}
PAIR_KINDS = {"absolute": 0, "delta": 1, "extrap": 2}


def pd_net_workspace_size(max_nodes):
    n = C.c_size_t(0)
    _check(None, _lib().pd_net_workspace_size(int(max_nodes), C.byref(n)), "pd_net_workspace_size")
    return n.value


def pd_net_create(max_nodes, ws_ptr, nbytes, stream_ptr):
    h = P()
    _check(None, _lib().pd_net_create(int(max_nodes), P(ws_ptr), int(nbytes), P(stream_ptr), C.byref(h)),
           "pd_net_create")
    return h


def pd_net_destroy(h):
    _lib().pd_net_destroy(h)


def _net_check(h, r, what):
    if r != 0:
        raise PdError(f"{what}: {STATUS.get(r, r)}")


def pd_net_set_params(h, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != PD_NET_NPARAMS:
        raise ValueError("need PD_NET_NPARAMS parameters")
    _net_check(h, _lib().pd_net_set_params(h, _ptr(a)), "pd_net_set_params")


def pd_net_get_params(h):
    a = np.zeros(PD_NET_NPARAMS, np.float32)
    _net_check(h, _lib().pd_net_get_params(h, _ptr(a)), "pd_net_get_params")
    return a


def pd_net_forward(h, x_ptr, B, H, W, y_ptr):
    _net_check(h, _lib().pd_net_forward(h, P(x_ptr), int(B), int(H), int(W), P(y_ptr)), "pd_net_forward")


def pd_net_loss_grad(h, x_ptr, t_ptr, B, H, W, want_loss=True, want_grads=False):
    loss = C.c_double(0.0)
    g = np.zeros(PD_NET_NPARAMS, np.float32) if want_grads else None
    _net_check(h, _lib().pd_net_loss_grad(h, P(x_ptr), P(t_ptr), int(B), int(H), int(W),
                                         C.byref(loss) if want_loss else None,
                                         _ptr(g) if want_grads else None), "pd_net_loss_grad")
    return (loss.value if want_loss else None), g


def pd_net_loss_grad_rz(h, x_ptr, B, H, W, want_loss=True, want_grads=False):
    loss = C.c_double(0.0)
    g = np.zeros(PD_NET_NPARAMS, np.float32) if want_grads else None
    _net_check(h, _lib().pd_net_loss_grad_rz(h, P(x_ptr), int(B), int(H), int(W),
                                            C.byref(loss) if want_loss else None,
                                            _ptr(g) if want_grads else None), "pd_net_loss_grad_rz")
    return (loss.value if want_loss else None), g


def pd_net_adam(h, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    _net_check(h, _lib().pd_net_adam(h, float(lr), float(b1), float(b2), float(eps)), "pd_net_adam")


def pd_warmstart_pairs(h, kind, x_ptr, t_ptr):
    k = PAIR_KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(h, _lib().pd_warmstart_pairs(h, k, P(x_ptr), P(t_ptr)), "pd_warmstart_pairs")


def pd_set_warm_start(h, mode, net_h=None):
    m = WARM_MODES[mode] if isinstance(mode, str) else int(mode)
    _check(h, _lib().pd_set_warm_start(h, m, net_h), "pd_set_warm_start")


def pd_get_rho(h, nodes):
    a = np.zeros(nodes, np.int64)
    b = np.zeros(nodes, np.int64)
    _check(h, _lib().pd_get_rho(h, _ptr(a), _ptr(b)), "pd_get_rho")
    return a, b


def pd_get_phi(h, nodes):
    a = np.zeros(nodes)
    _check(h, _lib().pd_get_phi(h, _dp(a)), "pd_get_phi")
    return a


def pd_get_field(h, nodes):
    a = np.zeros(nodes)
    b = np.zeros(nodes)
    _check(h, _lib().pd_get_field(h, _dp(a), _dp(b)), "pd_get_field")
    return a, b


def pd_get_density_map(h, species, nodes):
    a = np.zeros(nodes)
    _check(h, _lib().pd_get_density_map(h, int(species), _dp(a)), "pd_get_density_map")
    return a


def pd_get_energy_spectrum(h, species, lo, hi, nbins):
    a = np.zeros(nbins, np.uint64)
    _check(h, _lib().pd_get_energy_spectrum(h, int(species), float(lo), float(hi), int(nbins), _ptr(a)),
           "pd_get_energy_spectrum")
    return a


def pd_profile_enable(h, on):
    _check(h, _lib().pd_profile_enable(h, int(on)), "pd_profile_enable")


def pd_profile_read(h):
    ms = np.zeros(PD_NKERNELS)
    n = np.zeros(PD_NKERNELS, np.uint64)
    _check(h, _lib().pd_profile_read(h, _dp(ms), _ptr(n)), "pd_profile_read")
    return {pd_kernel_name(k): (float(ms[k]), int(n[k])) for k in range(PD_NKERNELS)}


def pd_kernel_name(k):
    return _lib().pd_kernel_name(int(k)).decode()


KERNEL_NAMES = ["inject", "push", "scan_bins", "scatter", "ncand", "scan_cand", "collide", "finalize",
                "poisson", "efield", "memset", "other", "coulomb"]


def pd_last_error(h):
    return _lib().pd_last_error(h).decode()


def pd_destroy(h):
    _lib().pd_destroy(h)


def pd_spectrum_static_max_bins():
    return int(_lib().pd_spectrum_static_max_bins())


def pd_energy_spectrum_static(key_ptr, vz_ptr, vr_ptr, vt_ptr, n, species, lo, hi, nbins, stream_ptr=0):
    """Energy histogram of raw device particle arrays (device pointers as ints),
    with no allocation; see include/pd.h for the shared-scratch rules."""
    if not 1 <= int(nbins) <= pd_spectrum_static_max_bins():
        raise PdError(f"pd_energy_spectrum_static: nbins = {nbins} is outside 1..{pd_spectrum_static_max_bins()}")
    a = np.zeros(nbins, np.uint64)
    r = _lib().pd_energy_spectrum_static(P(key_ptr), P(vz_ptr), P(vr_ptr), P(vt_ptr), int(n), int(species),
                                         float(lo), float(hi), int(nbins), P(stream_ptr), _ptr(a))
    _check(None, r, "pd_energy_spectrum_static")
    return a


class Net:
    """The warm-start network (pd_net) in a torch-allocated device workspace."""

    def __init__(self, max_nodes, params=None, device="cuda", stream=None):
        import torch
        load_library()
        self.max_nodes = int(max_nodes)
        self.nbytes = pd_net_workspace_size(self.max_nodes)
        self.ws = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.ws.device)
        self.h = pd_net_create(self.max_nodes, self.ws.data_ptr(), self.nbytes, self.stream.cuda_stream)
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        pd_net_set_params(self.h, params)

    def params(self):
        return pd_net_get_params(self.h)

    def forward(self, x):
        """x: torch CUDA float tensor [B, H, W] -> y (same shape)."""
        import torch
        x = x.contiguous()
        y = torch.empty_like(x)
        B, H, W = x.shape
        pd_net_forward(self.h, x.data_ptr(), B, H, W, y.data_ptr())
        return y

    def loss_grad(self, x, t, want_grads=False):
        x, t = x.contiguous(), t.contiguous()
        B, H, W = x.shape
        return pd_net_loss_grad(self.h, x.data_ptr(), t.data_ptr(), B, H, W, True, want_grads)

    def loss_grad_rz(self, x, want_grads=False):
        x = x.contiguous()
        B, H, W = x.shape
        return pd_net_loss_grad_rz(self.h, x.data_ptr(), B, H, W, True, want_grads)

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        pd_net_adam(self.h, lr, b1, b2, eps)

    def close(self):
        if getattr(self, "h", None):
            pd_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """A pd_sim in a torch-allocated device workspace on a torch stream."""

    def __init__(self, cfg_dict, xs=None, device="cuda", stream=None):
        import torch
        load_library()
        self.cfg_dict = dict(cfg_dict)
        self.cfg = config_from_dict(cfg_dict)
        self.nbytes = pd_workspace_size(self.cfg)
        self.ws = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.ws.device)
        self.h = pd_create(self.cfg, self.ws.data_ptr(), self.nbytes, self.stream.cuda_stream)
        rz = cfg_dict["geometry"] == "rz"
        self.nzn = cfg_dict["nz"] + (1 if rz else 0)
        self.nrn = cfg_dict["nr"] + (1 if rz else 0)
        self.nodes = self.nzn * self.nrn
        if xs is not None:
            self.set_cross_sections(xs)

    def set_cross_sections(self, xs):
        for ch, (E, s, th) in xs.items():
            pd_set_cross_section(self.h, ch, E, s, th)

    def set_sputter_yield(self, E, Y):
        pd_set_sputter_yield(self.h, E, Y)

    def load(self, parts):
        pd_load_particles(self.h, parts)

    def load_device(self, t):
        """t: dict of torch CUDA tensors (species u8, iz, ir i32, pz, pr, vz, vr, vt f32)."""
        keys = ("species", "iz", "ir", "pz", "pr", "vz", "vr", "vt")
        pd_load_particles_device(self.h, t["species"].numel(), [t[k].data_ptr() for k in keys])

    def set_field(self, Ez, Er):
        pd_set_field(self.h, Ez, Er)

    def step(self, n=1):
        pd_step(self.h, n)

    def synchronize(self):
        pd_synchronize(self.h)

    def scalars(self):
        return pd_get_scalars(self.h)

    def set_graph_mode(self, enable, poisson_cycles=4):
        pd_set_graph_mode(self.h, enable, poisson_cycles)

    def tuning(self):
        return pd_get_tuning(self.h)

    def save(self, path):
        pd_save(self.h, path)

    def warmstart_pairs(self, kind="absolute"):
        """(x, t) training pairs ("absolute", "delta" or "extrap") of the latest solves
        as torch CUDA tensors over all nodes (runs end to end)."""
        import torch
        x = torch.empty(self.nodes, dtype=torch.float32, device=self.ws.device)
        t = torch.empty(self.nodes, dtype=torch.float32, device=self.ws.device)
        pd_warmstart_pairs(self.h, kind, x.data_ptr(), t.data_ptr())
        return x, t

    def set_warm_start(self, mode, net=None):
        self._warm_net = net          # keep the network alive while it is in use
        pd_set_warm_start(self.h, mode, net.h if net is not None else None)

    def restore(self, path):
        pd_load(self.h, path)

    def rho_phi(self):
        """Node charge density (C/m^3) and potential (V), the Poisson training pairs."""
        return pd_get_rho_phi(self.h, self.nodes)

    def set_tuning(self, **kw):
        pd_set_tuning(self.h, **kw)

    def autotune(self, steps_per_trial=2):
        return pd_autotune(self.h, steps_per_trial)

    def counters(self):
        return pd_get_counters(self.h)

    def sort_stats(self):
        return pd_get_sort_stats(self.h)

    def bins(self):
        return pd_get_bins(self.h)

    def particles(self, live_only=True):
        return pd_get_particles(self.h, live_only)

    def rho(self):
        a, b = pd_get_rho(self.h, self.nodes)
        return a.reshape(self.nzn, self.nrn), b.reshape(self.nzn, self.nrn)

    def phi(self):
        return pd_get_phi(self.h, self.nodes).reshape(self.nzn, self.nrn)

    def field(self):
        a, b = pd_get_field(self.h, self.nodes)
        return a.reshape(self.nzn, self.nrn), b.reshape(self.nzn, self.nrn)

    def density_map(self, species):
        return pd_get_density_map(self.h, species, self.nodes).reshape(self.nzn, self.nrn)

    def energy_spectrum(self, species, lo=0.0, hi=500.0, nbins=100):
        return pd_get_energy_spectrum(self.h, species, lo, hi, nbins)

    def close(self):
        if getattr(self, "h", None):
            pd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble(Simulation):
    """Several independent runs advanced together (one launch per kernel for
    all runs).  `cfg_dicts` is a list of run configurations."""

    def __init__(self, cfg_dicts, xs=None, device="cuda", stream=None):
        import torch
        load_library()
        self.cfg_dicts = [dict(c) for c in cfg_dicts]
        self.cfg_dict = self.cfg_dicts[0]
        self.cfgs = [config_from_dict(c) for c in cfg_dicts]
        self.nbytes = pd_ensemble_workspace_size(self.cfgs)
        self.ws = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.ws.device)
        self.h = pd_ensemble_create(self.cfgs, self.ws.data_ptr(), self.nbytes, self.stream.cuda_stream)
        self.R = len(cfg_dicts)
        self.run_nodes = []
        for c in cfg_dicts:
            rz = c["geometry"] == "rz"
            self.run_nodes.append(((c["nz"] + (1 if rz else 0)), (c["nr"] + (1 if rz else 0))))
        self.nodes = sum(a * b for a, b in self.run_nodes)
        self.nzn, self.nrn = self.run_nodes[0]
        if xs is not None:
            self.set_cross_sections(xs)

    def load_run(self, run, parts):
        pd_load_particles_run(self.h, run, parts)

    def load_run_device(self, run, t):
        keys = ("species", "iz", "ir", "pz", "pr", "vz", "vr", "vt")
        pd_load_particles_device_run(self.h, run, t["species"].numel(), [t[k].data_ptr() for k in keys])

    def run_scalars(self, run):
        return pd_ensemble_get_scalars(self.h, run)

    def run_counters(self, run):
        return pd_get_run_counters(self.h, run)

    def run_slice(self, arr, run):
        """The part of a concatenated node array (rho, phi, field) that belongs to one run."""
        _, nb = pd_run_layout(self.h, run)
        a, b = self.run_nodes[run]
        return np.asarray(arr).ravel()[nb:nb + a * b].reshape(a, b)

    def run_density_map(self, run, species):
        a, b = self.run_nodes[run]
        return pd_get_run_density_map(self.h, run, species, a * b).reshape(a, b)

    def run_energy_spectrum(self, run, species, lo=0.0, hi=500.0, nbins=100):
        return pd_get_run_energy_spectrum(self.h, run, species, lo, hi, nbins)

    def rho(self):
        return pd_get_rho(self.h, self.nodes)

    def phi(self):
        return pd_get_phi(self.h, self.nodes)

    def field(self):
        return pd_get_field(self.h, self.nodes)

