"""Workload recipes (seeded, synthetic) shaped like the paper's runs.

Every function returns plain numpy arrays / dicts.  Particle loads are given in
the cell-relative form both implementations store: integer cell index along z
and r plus the offset inside the cell in [0, 1) as float32, and the three
velocity components (v_z, v_r, v_theta) in m/s as float32.

Species codes (the paper tracks e, Cu, Cu+, Cu2+ and labels Cu2+ by the channel
that made it, Sec. 2.3):
    0 = e, 1 = Cu, 2 = Cu+, 3 = Cu2+ made by step-wise Cu+ -> Cu2+ (label SW),
    4 = Cu2+ made by double ionization Cu -> Cu2+ (label DI).
"""
import math
import numpy as np

SPECIES = {"e": 0, "Cu": 1, "Cu+": 2, "Cu2+SW": 3, "Cu2+DI": 4, "Cu3+": 5, "Cu4+": 6}
SPECIES_NAMES = ["e", "Cu", "Cu+", "Cu2+SW", "Cu2+DI", "Cu3+", "Cu4+"]

# CODATA values, used here only to draw thermal velocities of the inputs.
_QE = 1.602176634e-19
_ME = 9.1093837015e-31
_KB = 1.380649e-23
_AMU = 1.66053906660e-27
_MCU = 63.546 * _AMU

# Cross-section grid: exponent-bucketed, XS_SUB points per octave from
# 2**XS_EMIN_EXP eV over XS_OCTAVES octaves (1e-3 .. 3.3e4 eV).
XS_EMIN_EXP = -10
XS_OCTAVES = 25
XS_SUB = 64


def xs_grid():
    """Energies (eV, float64, exactly representable in float32) of the table grid."""
    k = np.arange(XS_OCTAVES * XS_SUB + 1)
    e = XS_EMIN_EXP + k // XS_SUB
    j = k % XS_SUB
    return np.ldexp(1.0 + j / XS_SUB, e)


def standin_cross_sections(thresholds=None, peaks=None, sigma_el=5e-20, e_el=10.0, s_cx=6e-19, k_cx=0.06,
                           d_cu=2.6e-10):
    """Closed-form stand-ins for the paper's cross sections (its Fig. 1 data
    from refs. [28-30] is not available).  Ionization and excitation use the
    Lotz form with b = 0, sigma = s_max * e * ln(E/I) / (E/I) for E > I (peak
    s_max at E = e*I); elastic is sigma_el below e_el and falls as
    sqrt(e_el/E) above.  Returns {channel: (E_eV, sigma_m2, threshold_eV)} on
    the table grid.

    Channels: 0 elastic e-Cu, 1 excitation e-Cu, 2 single ionization Cu->Cu+,
    3 double ionization Cu->Cu2+, 4 step-wise Cu+->Cu2+, and the heavy pairs
    the paper lists without data: 5 resonant charge exchange Cu+ + Cu,
    sigma = s_cx (1 - k ln(E / 1 eV))^2 (the Rapp-Francis shape), and 6
    elastic Cu + Cu, a hard sphere pi d^2 (E: relative energy in the centre
    of mass, eV); 7 step-wise Cu2+ -> Cu3+ and 8 Cu3+ -> Cu4+ (Lotz, with the
    third and fourth ionization energies of Cu, 36.841 and 57.38 eV, which
    the paper does not give).
    Thresholds: DI about 28 eV and Cu+->Cu2+ 20.3 eV are the paper's (Sec. 3.2);
    7.726 eV (first ionization energy of Cu) and 3.8 eV (excitation) are not
    given by the paper.
    """
    th = {1: 3.8, 2: 7.726, 3: 28.0, 4: 20.3, 7: 36.841, 8: 57.38}
    pk = {1: 1.0e-20, 2: 3.0e-20, 3: 1.0e-21, 4: 1.5e-20, 7: 8.0e-21, 8: 5.0e-21}
    if thresholds:
        th.update(thresholds)
    if peaks:
        pk.update(peaks)
    E = xs_grid()
    out = {}
    s_el = np.where(E <= e_el, sigma_el, sigma_el * np.sqrt(e_el / np.maximum(E, 1e-300)))
    out[0] = (E, s_el, 0.0)
    for c in (1, 2, 3, 4, 7, 8):
        I = th[c]
        x = E / I
        s = np.where(x > 1.0, pk[c] * math.e * np.log(np.maximum(x, 1.0)) / x, 0.0)
        out[c] = (E, s, I)
    out[5] = (E, s_cx * np.maximum(1.0 - k_cx * np.log(E), 0.0) ** 2, 0.0)
    out[6] = (E, np.full_like(E, math.pi * d_cu * d_cu), 0.0)
    return out


def standin_sputter_yield(e_th=25.0, y0=2.0, power=2.5):
    """A stand-in for the ion-impact sputtering yield of Cu on Cu (the paper
    takes it from Yamamura and Tawara [32], whose formula and fitted
    parameters are not available): Y(E) = y0 (1 - sqrt(e_th / E))^power above
    the threshold e_th (eV), 0 below.  Returns (E_eV, Y) on the table grid."""
    E = xs_grid()
    Y = np.where(E > e_th, y0 * np.clip(1.0 - np.sqrt(e_th / E), 0.0, None) ** power, 0.0)
    return E, Y


def base_config(**kw):
    """Run parameters shared by every workload (the paper's Sec. 2.3 values
    where it gives them)."""
    c = dict(
        geometry="rz",          # "rz" (cylindrical, electrodes at z=0, z=L) or "xy_periodic"
        nz=64, nr=64,
        dz=6e-6 / 64, dr=6e-6 / 64,
        depth=1.0,              # Cartesian cell depth (m); unused in r-z
        dt=1e-15,               # electron step, 1 fs
        heavy_subcycle=10,      # heavy step = 10 electron steps
        weight=100.0,           # super-particle weight W
        seed=1, run=0,
        field_on=1, inject_on=1, di_on=1,
        V0=2.9e3, R_ohm=1e3, C_farad=1e-12,
        beta=35.0, tip_radius=100e-9, work_function=4.5,
        neutral_ratio=0.03, neutral_T=2000.0,
        capacity=1 << 16,
        max_cand_per_step=1 << 16,
        poisson_tol=1e-8,
    )
    c.update(kw)
    return c


def _maxwell(rng, n, sigma):
    return (rng.standard_normal((3, n)) * sigma).astype(np.float32)


def _uniform_pos(rng, n):
    # float32 offsets in [0, 1) with 24-bit resolution
    return (rng.integers(0, 1 << 24, size=(2, n), dtype=np.int64).astype(np.float64)
            * 2.0 ** -24).astype(np.float32)


def _load(cell_z, cell_r, rng, vsig, species):
    n = cell_z.size
    p = _uniform_pos(rng, n)
    if np.ndim(vsig) == 0:
        v = _maxwell(rng, n, vsig)
    else:
        v = (rng.standard_normal((3, n)) * vsig[None, :]).astype(np.float32)
    return dict(species=np.full(n, species, np.uint8),
                iz=cell_z.astype(np.int32), ir=cell_r.astype(np.int32),
                pz=p[0], pr=p[1], vz=v[0], vr=v[1], vt=v[2])


def concat_loads(loads):
    keys = ["species", "iz", "ir", "pz", "pr", "vz", "vr", "vt"]
    return {k: np.concatenate([l[k] for l in loads]) for k in keys}


def microbench(nz=1024, nr=1024, total=1e8, seed=1, dt=1e-15, coll_scale=1.0,
               Te_range=(5.0, 50.0), T_heavy=2000.0):
    """DSMC collision microbench: Cartesian nz x nr cells of 50 nm with
    periodic walls and no field.  Cu density per cell lognormal(ln 1e23 m^-3,
    1); Cu+ = 10 % of Cu; electrons = Cu+ (quasi-neutral); electron
    temperature per cell uniform in [5, 50] eV; heavies at 2000 K.  The cell
    depth is chosen so the expected particle total is `total`.
    `coll_scale` multiplies the collision time step only (stress variant)."""
    rng = np.random.default_rng(seed)
    ncell = nz * nr
    d = 50e-9
    mean_n = 1e23 * math.exp(0.5)
    W = 100.0
    # expected total = ncell * mean_n * V / W * (1 + 0.1 + 0.1)
    V = total * W / (ncell * mean_n * 1.2)
    depth = V / (d * d)
    n_cu = np.exp(math.log(1e23) + rng.standard_normal(ncell))
    N_cu = np.rint(n_cu * V / W).astype(np.int64)
    N_ion = np.rint(0.1 * N_cu).astype(np.int64)
    N_e = N_ion.copy()
    Te = rng.uniform(Te_range[0], Te_range[1], ncell)
    cells = np.arange(ncell, dtype=np.int64)
    loads = []
    for sp, N in ((0, N_e), (1, N_cu), (2, N_ion)):
        cidx = np.repeat(cells, N)
        if sp == 0:
            vsig = np.sqrt(Te[cidx] * _QE / _ME)
        else:
            vsig = math.sqrt(_KB * T_heavy / _MCU)
        loads.append(_load(cidx // nr, cidx % nr, rng, vsig, sp))
    cfg = base_config(geometry="xy_periodic", nz=nz, nr=nr, dz=d, dr=d, depth=depth,
                      dt=dt, heavy_subcycle=1, weight=W, seed=seed, field_on=0,
                      inject_on=0, di_on=1, coll_dt_scale=coll_scale,
                      capacity=int(1.02 * total) + (1 << 20))
    return cfg, concat_loads(loads)


def rz_breakdown(n=64, seed=1, di_on=1, capacity=20000):
    """Small Cu breakdown (r-z): n x n cells over the 6 um gap, planar
    electrodes, starting from vacuum (Sec. 2.3); FN electrons and 3 %
    neutrals are injected at the 200 nm tip each step."""
    d = 6e-6 / n
    cfg = base_config(geometry="rz", nz=n, nr=n, dz=d, dr=d, seed=seed, di_on=di_on,
                      capacity=capacity, max_cand_per_step=1 << 14)
    empty = concat_loads([_load(np.zeros(0, np.int64), np.zeros(0, np.int64),
                                np.random.default_rng(seed), 1.0, 0)])
    return cfg, empty


def rz_plume(n=512, total=2e7, seed=1, n0=1e26, lam=1e-6, rho0=1e-6, Te_eV=5.0,
             T_heavy=2000.0, capacity=None):
    """Production-size r-z breakdown snapshot: a near-cathode Cu plume
    n(z, r) = n0 exp(-z/lam) exp(-(r/rho0)^2), 60 % ionized with mean charge 2
    (Sec. 3.1: gamma ~ 60 %, Q ~ 2.0 in the burn), Cu2+ split SW:DI = 10:1,
    quasi-neutral electrons at Te.  The weight is scaled so the expected
    particle total is `total`."""
    rng = np.random.default_rng(seed)
    d = 6e-6 / n
    zc = (np.arange(n) + 0.5) * d
    rc = (np.arange(n) + 0.5) * d
    dens = n0 * np.exp(-zc / lam)[:, None] * np.exp(-(rc / rho0) ** 2)[None, :]
    vol = (np.pi * ((np.arange(n) + 1.0) ** 2 - np.arange(n) ** 2) * d * d * d)[None, :]
    heavy = dens * vol                     # physical heavy count per cell
    # heavies: 40 % Cu, 60 % Cu2+ (SW:DI = 10:1); electrons = 2 * Cu2+
    per_cell_particles = heavy * (0.4 + 0.6 + 1.2)
    W = float(per_cell_particles.sum() / total)
    cells = np.arange(n * n, dtype=np.int64)
    lam_cu = (0.4 * heavy / W).ravel()
    lam_sw = (0.6 * heavy / W * 10.0 / 11.0).ravel()
    lam_di = (0.6 * heavy / W * 1.0 / 11.0).ravel()
    N_cu = rng.poisson(lam_cu)
    N_sw = rng.poisson(lam_sw)
    N_di = rng.poisson(lam_di)
    N_e = 2 * (N_sw + N_di)
    vh = math.sqrt(_KB * T_heavy / _MCU)
    ve = math.sqrt(Te_eV * _QE / _ME)
    loads = []
    for sp, N, vs in ((0, N_e, ve), (1, N_cu, vh), (3, N_sw, vh), (4, N_di, vh)):
        cidx = np.repeat(cells, N)
        loads.append(_load(cidx // n, cidx % n, rng, vs, sp))
    if capacity is None:
        capacity = int(1.25 * total) + (1 << 20)
    cfg = base_config(geometry="rz", nz=n, nr=n, dz=d, dr=d, weight=W, seed=seed,
                      capacity=capacity, max_cand_per_step=1 << 22)
    return cfg, concat_loads(loads)


def rate_cell(n_e=200000, n_t=100000, Te_eV=10.0, seed=3, depth=1e-6, dt=1e-15,
              coll_scale=1.0, target_species=1, ncells=1):
    """Frozen-target rate check input: `ncells` Cartesian cells holding
    Maxwellian electrons at Te and cold targets (zero velocity), so that the
    DSMC operator reduces to the linear test-particle (MCC) one of Eq. (3)."""
    rng = np.random.default_rng(seed)
    d = 50e-9
    ve = math.sqrt(Te_eV * _QE / _ME)
    ce = rng.integers(0, ncells, n_e)
    ct = rng.integers(0, ncells, n_t)
    le = _load(np.zeros(n_e, np.int64), ce, rng, ve, 0)
    lt = _load(np.zeros(n_t, np.int64), ct, rng, 0.0, target_species)
    lt["vz"][:] = 0
    lt["vr"][:] = 0
    lt["vt"][:] = 0
    cfg = base_config(geometry="xy_periodic", nz=1, nr=ncells, dz=d, dr=d, depth=depth,
                      dt=dt, heavy_subcycle=1, weight=100.0, seed=seed, field_on=0,
                      inject_on=0, coll_dt_scale=coll_scale,
                      capacity=n_e * 3 + n_t + (1 << 16), max_cand_per_step=1 << 22)
    return cfg, concat_loads([le, lt])


def heavy_cells(n_e=3000, n_cu=6000, n_cup=1500, ncells=4, Te_eV=30.0, T_heavy=2000.0, seed=9,
                coll_scale=1.0, heavy_coll=1, depth=1e-6, dt=1e-15, capacity=1 << 21):
    """Dense Cartesian cells (a 2 x ncells grid, the second row empty) of
    Maxwellian electrons at Te and Maxwellian Cu and Cu+ at T_heavy, spread
    uniformly over the first row's cells: every step is a heavy step, so the
    heavy-particle pair classes run beside the electron ones.  The capacity
    leaves room for the slots that candidates of the electron classes reserve
    (two each, per step)."""
    rng = np.random.default_rng(seed)
    d = 50e-9
    ve = math.sqrt(Te_eV * _QE / _ME)
    vh = math.sqrt(_KB * T_heavy / _MCU)
    loads = []
    for sp, n, vs in ((0, n_e, ve), (1, n_cu, vh), (2, n_cup, vh)):
        loads.append(_load(np.zeros(n, np.int64), rng.integers(0, ncells, n), rng, vs, sp))
    cfg = base_config(geometry="xy_periodic", nz=2, nr=max(2, ncells), dz=d, dr=d, depth=depth,
                      dt=dt, heavy_subcycle=1, weight=100.0, seed=seed, field_on=0,
                      inject_on=0, coll_dt_scale=coll_scale, heavy_coll=heavy_coll,
                      capacity=capacity, max_cand_per_step=1 << 22)
    return cfg, concat_loads(loads)


ENSEMBLE_GRIDS = (64, 96, 128, 192, 256)
ENSEMBLE_VOLTS_KV = (2.0, 3.0, 4.0, 5.0, 6.0, 7.0, 8.0, 10.0)


def ensemble_breakdown(seeds=range(1, 9), volts_kV=ENSEMBLE_VOLTS_KV, grids=ENSEMBLE_GRIDS,
                       n_lo=1e5, n_hi=2e6, emission=False):
    """Ensemble of independent breakdown runs, seeds x gap voltages (run index
    = seed position * len(volts_kV) + voltage position).  Each run draws, from
    a numpy Philox generator keyed by its run index, its grid N (N x N cells,
    one of `grids`) and its particle count, log-uniform in [n_lo, n_hi]; its
    initial load is the near-cathode plume of `rz_plume` scaled to that grid
    and count.  Field: the self-consistent Poisson solve.  Cathode emission is
    off unless `emission`: the plume's charge noise puts 1e10-1e11 V/m on the
    cathode, and with the tip enhancement of 35 the Fowler-Nordheim count per
    step then outgrows any capacity within a few steps on the coarser runs.
    Returns a list of (config, particles)."""
    out = []
    seeds = list(seeds)
    for si, seed in enumerate(seeds):
        for vi, kv in enumerate(volts_kV):
            run = si * len(volts_kV) + vi
            pick = np.random.Generator(np.random.Philox(key=run))
            n = int(grids[int(pick.integers(0, len(grids)))])
            count = float(math.exp(pick.uniform(math.log(n_lo), math.log(n_hi))))
            cfg, parts = rz_plume(n=n, total=count, seed=1000 * int(seed) + run)
            cfg.update(seed=int(seed), run=run, V0=kv * 1e3, field_on=1, inject_on=int(bool(emission)),
                       capacity=int(1.25 * count) + (1 << 16))
            out.append((cfg, parts))
    return out
