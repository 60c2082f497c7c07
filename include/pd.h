/*
 * pd.h -- C ABI of the GB300 PIC-DSMC particle pipeline.
 *
 * The library advances the 2D3V particle-in-cell / direct-simulation Monte
 * Carlo model of W. Yang et al., "The role of double ionization on the
 * generation of doubly charged ions in copper vacuum arcs" (arXiv:2109.00214):
 * electrons, Cu, Cu+ and Cu2+ super-particles (Cu2+ labelled by the channel
 * that made it, Sec. 2.3), electron-impact DSMC collisions with five channels
 * including the four-stage double-ionization scheme of Sec. 2.2, the
 * electrostatic push, fixed-point charge deposition (Eq. (9)-(10)) and the
 * Poisson solve (Eq. (8)).  Every step of the pipeline runs in this library's
 * CUDA kernels on the stream the caller supplies.
 *
 * Conventions
 *   - Every call returns pd_status; PD_OK is 0.  Nothing is thrown across
 *     the ABI.  After a failing call, pd_last_error() gives a message.
 *   - Kernels report failures (capacity exhausted, a bounded wait that ran
 *     out) through a sticky device error word; it is read at the next call
 *     that synchronises (pd_synchronize, pd_get_*), which then fails.
 *   - Ownership: the caller owns the device workspace (any device
 *     allocation, e.g. a torch tensor), the CUDA stream and every host
 *     buffer.  The library keeps only small host metadata, freed by
 *     pd_destroy.  It never allocates device memory itself.
 *   - Units are SI unless a name ends in _eV.  Geometry: axial index iz along
 *     z (cathode at z = 0, anode at z = L = nz dz), radial index ir along r
 *     (axis at r = 0); in the Cartesian periodic mode the same two indices
 *     are the two in-plane axes.  Cell index = iz * nr + ir.
 *   - Species codes: 0 e, 1 Cu, 2 Cu+, 3 Cu2+ from Cu+ -> Cu2+ (label SW),
 *     4 Cu2+ from Cu -> Cu2+ (label DI).  Channels: 0 elastic e-Cu,
 *     1 excitation e-Cu, 2 ionization Cu -> Cu+, 3 double ionization
 *     Cu -> Cu2+, 4 ionization Cu+ -> Cu2+.
 */
#ifndef PD_H
#define PD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PD_OK = 0,
    PD_ERR_ARG = 1,        /* invalid argument or configuration */
    PD_ERR_CAPACITY = 2,   /* particle capacity or id space exhausted */
    PD_ERR_CUDA = 3,       /* a CUDA runtime call failed */
    PD_ERR_TIMEOUT = 4,    /* reserved: a bounded device wait ran out (no kernel of this
                              version waits on another, so none reports it) */
    PD_ERR_NONFINITE = 5,  /* NaN/Inf met where a finite value is required */
    PD_ERR_STATE = 6       /* call not valid in the current state */
} pd_status;

enum { PD_GEOM_RZ = 0, PD_GEOM_XY_PERIODIC = 1 };
enum { PD_FIELD_NONE = 0, PD_FIELD_POISSON = 1, PD_FIELD_EXTERNAL = 2 };
/* species: Cu2+ carries the label of its route (step-wise or double
 * ionization, Sec. 2.3); Cu3+ and Cu4+ exist only with charge_max 3 and 4 */
enum { PD_SP_E = 0, PD_SP_CU = 1, PD_SP_CUP = 2, PD_SP_CU2_SW = 3, PD_SP_CU2_DI = 4, PD_SP_CU3 = 5,
       PD_SP_CU4 = 6, PD_NSP = 7 };
/* channels 5 and 6: the heavy pairs the paper lists besides ionization
 * (Sec. 2.3, no data given): resonant charge exchange Cu+ + Cu and elastic
 * Cu + Cu, with E the relative energy in the centre of mass; channels 7 and
 * 8: the step-wise ionizations Cu2+ -> Cu3+ (either Cu2+ label) and
 * Cu3+ -> Cu4+ (Sec. 2.3) */
enum { PD_CH_ELASTIC = 0, PD_CH_EXCITATION = 1, PD_CH_SI = 2, PD_CH_DI = 3, PD_CH_SW = 4,
       PD_CH_CX = 5, PD_CH_NN = 6, PD_CH_S3 = 7, PD_CH_S4 = 8, PD_NCH = 9 };

#define PD_CONFIG_VERSION 4u

/* Run parameters (Sec. 2.3 gives: 50 nm cells, 1 fs electron step, heavy step
 * ten times longer, W = 100, 2.9 kV through R = 1 kOhm with C = 1 pF, a 200 nm
 * tip with field enhancement 35, neutral flux 3 % of the electron flux). */
typedef struct pd_config {
    uint32_t struct_size;      /* sizeof(pd_config); checked */
    uint32_t version;          /* PD_CONFIG_VERSION */
    int32_t geometry;          /* PD_GEOM_* */
    int32_t nz, nr;            /* cells along z and r; nz * nr < 2^24 */
    double dz, dr;             /* cell size (m) */
    double depth;              /* Cartesian cell depth (m); unused in r-z */
    double dt;                 /* electron time step (s) */
    int32_t heavy_subcycle;    /* heavies move every this many electron steps */
    double weight;             /* physical particles per super-particle */
    uint32_t seed, run;        /* Philox key */
    int32_t field_mode;        /* PD_FIELD_*; PD_FIELD_POISSON needs r-z */
    int32_t inject_on;         /* cathode emission each step (r-z only) */
    int32_t di_on;             /* double-ionization channel on */
    int32_t di_split_mode;     /* 0: cos chi = R, 1: cos^2 chi = R (stage 4) */
    double coll_dt_scale;      /* collision time step / electron time step */
    double V0, R_ohm, C_farad; /* external circuit */
    double beta, tip_radius, work_function, neutral_ratio, neutral_T;
    double poisson_tol;        /* relative residual |b - A phi| / |b| */
    int32_t poisson_max_cycles;
    int32_t heavy_coll;        /* 1: on heavy steps, the heavy pair classes (Cu+, Cu)
                                  charge exchange and (Cu, Cu) elastic, NTC with the
                                  heavy step; 0 (default): off */
    int32_t charge_max;        /* highest ion charge: 2 (default), 3 (adds the pair
                                  classes (e, Cu2+) -> Cu3+), 4 (and (e, Cu3+) -> Cu4+);
                                  species above it are refused on load */
    int32_t coulomb;           /* 1: Coulomb collisions of the e-e and e-ion pairs of
                                  each cell after its DSMC classes, and of its ion
                                  pairs on heavy steps (binary collision model of
                                  Takizuka and Abe); 0 (default): off */
    int64_t capacity;          /* particle slots */
    double coulomb_lnl;        /* Coulomb logarithm (default 10) */
    int32_t sputter;           /* 1: ions absorbed at an electrode sputter Cu atoms into
                                  the gap, floor(Y(E) + R) per ion super-particle (yield
                                  from pd_set_sputter_yield); 0 (default): off */
    int32_t reserved1;         /* 0 */
    double sputter_T;          /* temperature (K) of the sputtered atoms' effusive flux */
} pd_config;

/* Scalars of the current state (Sec. 3: arc current and voltage, Eq. (21)
 * ionization degree and mean charge, cathode erosion). */
typedef struct pd_scalars {
    double t;                  /* simulated time (s) */
    double V;                  /* anode voltage (V) */
    double I_gap;              /* gap current of the last step (A) */
    double gamma;              /* ionization degree, Eq. (21), all ion charges */
    double Qbar;               /* mean ion charge, Eq. (21) */
    double erosion;            /* cathode erosion: net Cu mass / charge (kg/C) */
    double mass;               /* net Cu mass leaving the cathode (kg) */
    double charge;             /* net charge through the cathode (C) */
    double sgmax[2];           /* NTC majorants (sigma g)_max, (e,Cu), (e,Cu+) */
    double poisson_relres;     /* last solve's relative residual */
    double poisson_cycles;     /* last solve's multigrid cycles */
    double poisson_relres_max; /* largest final relative residual of the solves
                                  issued by the latest pd_step call */
    double poisson_relres0;    /* last solve's relative residual at its start
                                  (the quality of the warm start) */
    double absorbed_energy[3]; /* J absorbed at cathode, anode, outer wall */
    int64_t n_particles;       /* live particles */
    int64_t count[PD_NSP];     /* live particles per species */
    int64_t step;              /* electron steps taken */
} pd_scalars;

/* counters: events of channels 0-4 [5], null candidates, candidates whose
 * target (or, for heavy pairs, either particle) was already ionized this
 * step, accepted candidates below threshold, NTC majorant violations,
 * isotropic-sampling fallbacks, candidates in total, electrons emitted,
 * neutrals emitted, absorbed [electrode 3][species 7], then events of charge
 * exchange, Cu-Cu elastic, Cu2+ -> Cu3+ and Cu3+ -> Cu4+, then Coulomb pair
 * collisions e-e and e-ion, then atoms sputtered from the cathode and from
 * the anode, then Coulomb ion-ion pair collisions. */
#define PD_NCOUNTERS 43

typedef struct pd_sim pd_sim;

/* Defaults: the paper's run parameters on a 64 x 64 r-z grid over the 6 um
 * gap (Sec. 2.3). */
pd_status pd_config_default(pd_config* cfg);

/* Device workspace bytes pd_create needs for cfg. */
pd_status pd_workspace_size(const pd_config* cfg, size_t* bytes);

/* Create a simulation in a caller-owned device workspace (at least
 * pd_workspace_size bytes, 256-byte aligned) on stream `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  The current CUDA device
 * must be the workspace's device.  The simulation starts empty (vacuum,
 * Sec. 2.3), with zero cross sections and no field. */
pd_status pd_create(const pd_config* cfg, void* dev_workspace, size_t bytes, void* cuda_stream,
                    pd_sim** out);

/* Integrated cross section of one channel (Sec. 2.3, Fig. 1 of the paper) as
 * n >= 2 points (E_eV ascending, sigma_m2) in host memory, copied.  The table
 * is resampled by linear interpolation onto the library's grid (64 points per
 * octave from 2^-10 eV to 2^15 eV) and is zero below threshold_eV, which is
 * also the energy the channel removes (Eq. (6), dE = -E_th).  Recomputes the
 * NTC majorants.  Synchronous with respect to the host. */
pd_status pd_set_cross_section(pd_sim* sim, int channel, const double* E_eV, const double* sigma_m2,
                               int n, double threshold_eV);

/* Ion-impact sputtering yield (Sec. 2.3; the paper's yield is that of
 * Yamamura and Tawara): Y(E) sputtered Cu atoms per ion arriving at an
 * electrode with kinetic energy E, as n >= 2 points (E_eV ascending, Y) in
 * host memory, copied and resampled like a cross section (no threshold: the
 * table carries its own).  Used when pd_config.sputter is 1; the default
 * table is zero.  Synchronous with respect to the host. */
pd_status pd_set_sputter_yield(pd_sim* sim, const double* E_eV, const double* Y, int n);

/* Append n particles given on the host in cell-relative form: species code,
 * cell indices iz, ir, offsets pz, pr in [0, 1) inside the cell, velocities
 * vz, vr, vt (m/s).  Ids are assigned in order.  Copied (synchronous). */
pd_status pd_load_particles(pd_sim* sim, int64_t n, const uint8_t* species, const int32_t* iz,
                            const int32_t* ir, const float* pz, const float* pr, const float* vz,
                            const float* vr, const float* vt);

/* Same, with all nine arrays in device memory (asynchronous on the stream;
 * the arrays must stay valid until the stream reaches the copy). */
pd_status pd_load_particles_device(pd_sim* sim, int64_t n, const uint8_t* species, const int32_t* iz,
                                   const int32_t* ir, const float* pz, const float* pr, const float* vz,
                                   const float* vr, const float* vt);

/* External node field (field_mode PD_FIELD_EXTERNAL), host arrays of
 * (nz+1)*(nr+1) nodes in r-z or nz*nr in the periodic mode, row-major in iz. */
pd_status pd_set_field(pd_sim* sim, const double* Ez, const double* Er);

/* Switch cathode emission (FN electrons + neutrals, Sec. 2.3) on or off. */
pd_status pd_inject_cathode(pd_sim* sim, int enable);

/* Advance n_steps electron steps: inject -> push + deposit -> sort ->
 * collide + spawn -> circuit -> Poisson -> E.  Asynchronous on the stream. */
pd_status pd_step(pd_sim* sim, int64_t n_steps);

/* Wait for the stream and report a device-side error if one was raised. */
pd_status pd_synchronize(pd_sim* sim);

/* Diagnostics (synchronise). */
pd_status pd_get_scalars(pd_sim* sim, pd_scalars* out);
pd_status pd_get_counters(pd_sim* sim, uint64_t* out /* PD_NCOUNTERS */);
/* Slots in use (live + dead); size for pd_get_particles. */
pd_status pd_particle_slots(pd_sim* sim, int64_t* slots);
/* State of the cell sort (no counterpart in the paper: the particle store's
 * bookkeeping).  Particles are kept in bins of one species and cell with
 * slack slots after each bin's particles; a step moves only the particles
 * that change bin, and lays all bins out anew (with slack sized from each
 * bin's traffic) only when a bin runs out of slots.  Synchronises. */
typedef struct pd_sort_stats {
    uint64_t relayouts;        /* new layouts of the bins since create (or load) */
    uint64_t bin_slots;        /* slots of all bins, live and slack */
    uint64_t live;             /* particles in bins */
    uint64_t steps_since;      /* steps since the last new layout */
    uint64_t faults;           /* consistency checks of the sort that failed (a bit per check), 0 if none */
} pd_sort_stats;
pd_status pd_get_sort_stats(pd_sim* sim, pd_sort_stats* out);
/* The bins of the sort (for tests and diagnostics): `start` (nbins + 1
 * entries, host) receives the first slot of each bin and, last, the first
 * slot of the tail; `count` (nbins entries, host) the particles of each bin.
 * Bins are species-major: bin = species * cells + cell, for the species that
 * have bins (5, or 7 with charge_max >= 3); *nbins receives their number when
 * `start` and `count` are NULL.  Synchronises. */
pd_status pd_get_bins(pd_sim* sim, uint32_t* start, uint32_t* count, int64_t* nbins);
/* Copy every slot to host arrays of pd_particle_slots() entries; dead slots
 * have species 255 and run -1.  Order is the device order (cell-sorted, not
 * by id).  `run` (may be NULL) receives the run of each particle; iz, ir are
 * local to that run. */
pd_status pd_get_particles(pd_sim* sim, uint32_t* id, int32_t* run, uint8_t* species, int32_t* iz, int32_t* ir,
                           float* pz, float* pr, float* vz, float* vr, float* vt);
/* Fixed-point node charge (units of e * 2^-32 per super-particle) of the
 * electrons and of the heavies. */
pd_status pd_get_rho(pd_sim* sim, int64_t* rho_e, int64_t* rho_h);
pd_status pd_get_phi(pd_sim* sim, double* phi);
/* Training pairs of the Poisson solve (Eq. (8)): node charge density
 * rho = e W (rho_e + rho_h) 2^-32 / V_node in C/m^3 (V_node: Verboncoeur's
 * node volumes in r-z, dz dr depth in the Cartesian mode) and the node
 * potential phi in V, both host arrays of all runs' nodes end to end. */
pd_status pd_get_rho_phi(pd_sim* sim, double* rho, double* phi);
pd_status pd_get_field(pd_sim* sim, double* Ez, double* Er);
/* Number density (m^-3) of one species on the nodes (CIC / node volume). */
pd_status pd_get_density_map(pd_sim* sim, int species, double* out);
/* Kinetic-energy histogram (eV) of one species on [e_lo_eV, e_hi_eV). */
pd_status pd_get_energy_spectrum(pd_sim* sim, int species, double e_lo_eV, double e_hi_eV, int nbins,
                                 uint64_t* out);

/* Per-kernel CUDA-event timing of the launches pd_step makes (for
 * measurement).  enable != 0 starts recording; pd_profile_read synchronises
 * and returns, per kernel id, total milliseconds and launch counts, then
 * clears.  Kernel ids: see pd_kernel_name. */
#define PD_NKERNELS 13
pd_status pd_profile_enable(pd_sim* sim, int enable);
pd_status pd_profile_read(pd_sim* sim, double* ms /* PD_NKERNELS */, uint64_t* launches /* PD_NKERNELS */);
const char* pd_kernel_name(int kernel_id);

const char* pd_last_error(const pd_sim* sim);
void pd_destroy(pd_sim* sim);

/* ---------------------------------------------------------------------
 * Ensembles: several independent breakdown runs (e.g. seeds x gap voltages,
 * each with its own grid, particle load, weight, circuit and emission)
 * advanced together.  Every kernel launch of a step covers all runs: their
 * cells and nodes are laid end to end in one index space (cells of run r
 * start at its cell_base, nodes at its node_base) and the particle store is
 * shared.  Each run evolves exactly as the same run would alone (its Philox
 * key is its own (seed, run) and draws are keyed by its local cells).  The
 * runs must agree on geometry, dt, heavy_subcycle, field_mode,
 * coll_dt_scale, di_on and di_split_mode; at most 128 runs and 2^24 cells in
 * total.  pd_sim functions apply to an ensemble (the single-run getters
 * report run 0; grids returned by pd_get_rho/phi/field are the runs' grids
 * end to end).
 * --------------------------------------------------------------------- */
typedef struct pd_sim pd_ensemble;
pd_status pd_ensemble_workspace_size(const pd_config* cfgs, int n_runs, size_t* bytes);
pd_status pd_ensemble_create(const pd_config* cfgs, int n_runs, void* dev_workspace, size_t bytes,
                             void* cuda_stream, pd_ensemble** out);
pd_status pd_ensemble_step(pd_ensemble* ens, int64_t n_steps);
pd_status pd_ensemble_get_scalars(pd_ensemble* ens, int run, pd_scalars* out);
pd_status pd_run_count(pd_sim* sim, int* n_runs);
/* first global cell and node of a run */
pd_status pd_run_layout(pd_sim* sim, int run, int64_t* cell_base, int64_t* node_base);
pd_status pd_get_run_counters(pd_sim* sim, int run, uint64_t* out /* PD_NCOUNTERS */);
pd_status pd_get_run_density_map(pd_sim* sim, int run, int species, double* out);
pd_status pd_get_run_energy_spectrum(pd_sim* sim, int run, int species, double e_lo_eV, double e_hi_eV,
                                     int nbins, uint64_t* out);
/* loads into one run (iz, ir local to the run); see pd_load_particles */
pd_status pd_load_particles_run(pd_sim* sim, int run, int64_t n, const uint8_t* species, const int32_t* iz,
                                const int32_t* ir, const float* pz, const float* pr, const float* vz,
                                const float* vr, const float* vt);
pd_status pd_load_particles_device_run(pd_sim* sim, int run, int64_t n, const uint8_t* species,
                                       const int32_t* iz, const int32_t* ir, const float* pz, const float* pr,
                                       const float* vz, const float* vr, const float* vt);

/* CUDA-graph stepping.  When enabled, pd_step captures G steps (G = the heavy
 * sub-cycle rounded up to an even number) once into a graph and replays it
 * with one launch per G steps; the step counter that keys the random streams
 * lives on the device, so replays draw fresh numbers.  The Poisson solve then
 * runs exactly `poisson_cycles` multigrid cycles per step with no host
 * synchronisation (runs that reach their tolerance earlier skip the rest);
 * the achieved residual is reported in pd_scalars.  Steps not aligned to G
 * run eagerly.  Changing cross sections or emission drops the graph. */
pd_status pd_set_graph_mode(pd_sim* sim, int enable, int poisson_cycles);

/* Launch shapes of the step's kernels.  Every one of these kernels walks its
 * work with a grid-stride loop and writes results that do not depend on the
 * order in which threads run (integer atomics, per-cell work, canonical id
 * order), so a shape changes speed only, never a result.  Grids are given
 * in blocks per SM (1..64); mg_threads is the block size of the multigrid
 * level kernels (a multiple of 32 in 64..1024) and mg_max_blocks caps their
 * blocks per run and level (1..65535).  pd_set_tuning validates and drops
 * a captured graph. */
typedef struct pd_tuning {
    int push_blocks_per_sm;     /* push + gather + deposit (256 threads) */
    int bincount_blocks_per_sm; /* sort: bin counts (256 threads) */
    int scatter_blocks_per_sm;  /* sort: scatter (256 threads) */
    int ncand_blocks_per_sm;    /* NTC candidate counts (256 threads) */
    int collide_blocks_per_sm;  /* collisions (128 threads) */
    int mg_threads;
    int mg_max_blocks;
} pd_tuning;
pd_status pd_get_tuning(pd_sim* sim, pd_tuning* out);
pd_status pd_set_tuning(pd_sim* sim, const pd_tuning* t);

/* Autotuner: picks each pd_tuning entry in turn (coordinate descent over a
 * fixed candidate list per entry) by timing its kernel with CUDA events over
 * `steps_per_trial` eager steps after one untimed step per candidate, keeps
 * the fastest and leaves it set; `out` (may be null) receives the choice.
 * The trial steps are real steps: the simulation advances by every step the
 * tuner takes (pd_scalars.step counts them).  steps_per_trial in 1..64.
 * Per-kernel profile records taken before the call are discarded. */
pd_status pd_autotune(pd_sim* sim, int steps_per_trial, pd_tuning* out);

/* Checkpoint and resume.  pd_save synchronises and writes the whole state of
 * a simulation or ensemble to a file: its configs, cross-section tables, the
 * particle slots in their sorted order with the bin offsets, node charge,
 * potential and field, every run's counters, ledgers and circuit state, and
 * the step counter.  pd_load reads such a file into a simulation created
 * with the same configs (compared field by field); pd_step then continues
 * exactly as the saved simulation would have, with bit-identical results.
 * Launch shapes, graph mode and profiling are not saved.  Errors: PD_ERR_ARG
 * for an unreadable, truncated or foreign file or different configs, and
 * PD_ERR_CAPACITY when the saved slots exceed the capacity; a failed load
 * can leave the simulation's state partly overwritten. */
pd_status pd_save(pd_sim* sim, const char* path);
pd_status pd_load(pd_sim* sim, const char* path);

/* ---- Learned warm start of the Poisson solve (Eq. (8)) -------------------
 *
 * A six-layer convolutional network predicts the potential from the charge
 * density so that the multigrid solve starts closer to its answer; the solve
 * still runs to the configured residual.  Node arrays of one r-z run are
 * (nz + 1) x (nr + 1); z_i = i dz, L = nz dz; rho in C/m^3 (Verboncoeur's
 * node volumes, halved on the electrode rows).  Three formulations:
 *   absolute (PD_WARM_LEARNED): d = rho, base = V z / L;
 *   delta (PD_WARM_LEARNED_DELTA): d = rho - rho', base = phi' + (V - V') z / L,
 *     where rho', phi', V' belong to the previous solve;
 *   extrapolated (PD_WARM_LEARNED_EXTRAP): d = rho - (2 rho' - rho''),
 *     base = 2 phi' - phi'' + (V - 2 V' + V'') z / L, with rho'', phi'', V''
 *     of the solve before the previous one: the network corrects the
 *     potential extrapolated linearly in time from the charge the
 *     extrapolation misses;
 * and, for all, with m = max |d| over the run's nodes:
 *   x = d / m  (x = 0 when m = 0)                       (network input)
 *   t = (phi - base) eps0 / (m dz^2)                    (training target)
 *   phi_0 = base + y m dz^2 / eps0                      (warm start from y ~ t)
 * (dz^2 makes t the potential in grid units of the unit-spacing Laplacian.)
 * Network: 3 x 3 convolutions, zero padding, channels 1 -> 32 -> 32 -> 32 ->
 * 32 -> 32 -> 1, ReLU after the first five, a bias per output channel.
 * Parameters (PD_NET_NPARAMS floats): for each layer in order its weights
 * W[tap][c_out][c_in], tap = 3 (dy + 1) + (dx + 1) for the input node at
 * (i + dy, j + dx), then its biases.  Layers compute with bfloat16 weights
 * and activations and float accumulation; the optimiser keeps float master
 * weights.  Loss: mean over samples and nodes of (y - t)^2 (pd_net_loss_grad),
 * or the residual of Eq. (8) that the start leaves (pd_net_loss_grad_rz);
 * optimiser: Adam. */
#define PD_NET_NPARAMS 37601
typedef struct pd_net pd_net;

/* Device workspace for a network that processes up to max_nodes nodes per
 * call (the sum over the samples of a batch of (nz + 1)(nr + 1)). */
pd_status pd_net_workspace_size(int64_t max_nodes, size_t* bytes);
pd_status pd_net_create(int64_t max_nodes, void* dev_workspace, size_t bytes, void* cuda_stream, pd_net** out);
void pd_net_destroy(pd_net* net);
/* Host float arrays of PD_NET_NPARAMS values; set resets the optimiser. */
pd_status pd_net_set_params(pd_net* net, const float* params);
pd_status pd_net_get_params(pd_net* net, float* params);
/* Inference on a batch of B samples of H x W nodes stored one after another
 * (x, y: device float arrays of B H W values). */
pd_status pd_net_forward(pd_net* net, const float* x, int B, int H, int W, float* y);
/* Forward and back-propagation of the loss against targets t (device,
 * B H W floats): *loss (host, may be null) receives the loss and grads
 * (host, PD_NET_NPARAMS floats, may be null) the gradient; the gradient is
 * also kept for pd_net_adam.  Synchronises when loss or grads is given. */
pd_status pd_net_loss_grad(pd_net* net, const float* x, const float* t, int B, int H, int W, double* loss,
                           float* grads);
/* The same with the residual loss of a start phi_0 = base + y m dz^2 /
 * eps0 on r-z grids with dz = dr: on the interior rows (1 .. H - 2; the
 * electrode rows are Dirichlet and y is not used there)
 *   r = w x - S y,
 *   (S y)_ij = (a+_j + a-_j + 2 w_j) y_ij - a+_j y_i,j+1 - a-_j y_i,j-1
 *              - w_j (y_i+1,j + y_i-1,j)   (y = 0 on rows 0 and H - 1),
 * the finite-volume equations of Eq. (8) divided by 2 pi dr^3 m / eps0, with
 * a+_j = j + 1/2 (0 at j = W - 1), a-_j = j - 1/2 (0 at j = 0), w_j = j,
 * 1/8 at j = 0 and (W - 1)/2 - 1/8 at j = W - 1 (the node's finite volume
 * over 2 pi dr^3); loss = sum of r^2 / (B (H - 2) W).  The target of the
 * pair is not needed: the exact t gives r = 0.  H >= 3, W >= 2. */
pd_status pd_net_loss_grad_rz(pd_net* net, const float* x, int B, int H, int W, double* loss, float* grads);
/* One Adam step (b1, b2, eps as in Kingma and Ba) with the gradient of the
 * last pd_net_loss_grad or pd_net_loss_grad_rz. */
pd_status pd_net_adam(pd_net* net, float lr, float b1, float b2, float eps);

/* Training pairs (x, t) of every run from the most recent solve (kind
 * PD_PAIRS_ABSOLUTE), the two most recent (PD_PAIRS_DELTA) or the three
 * most recent (PD_PAIRS_EXTRAP), written to device float arrays laid out
 * like the node arrays of pd_get_phi.  PD_ERR_STATE until enough solves have
 * run since the simulation was created or loaded. */
enum { PD_PAIRS_ABSOLUTE = 0, PD_PAIRS_DELTA = 1, PD_PAIRS_EXTRAP = 2 };
pd_status pd_warmstart_pairs(pd_sim* sim, int kind, float* x, float* t);

/* Starting point of each Poisson solve: PD_WARM_PREVIOUS (default: the
 * previous step's potential), PD_WARM_COLD (the charge-free potential
 * V z / L), PD_WARM_LEARNED, PD_WARM_LEARNED_DELTA or PD_WARM_LEARNED_EXTRAP
 * (phi_0 from `net`, which must stay alive and hold at least the
 * simulation's node count; the delta and extrapolated forms fall back to the
 * previous potential until one or two solves have been made since create or
 * load), PD_WARM_EXTRAPOLATE (linear in time through the two previous
 * solutions, 2 phi_{n-1} - phi_{n-2}, on the interior rows; the previous
 * potential until two solves have been made since create or load).  r-z
 * Poisson mode only.  Drops a captured graph. */
enum { PD_WARM_PREVIOUS = 0, PD_WARM_COLD = 1, PD_WARM_LEARNED = 2, PD_WARM_LEARNED_DELTA = 3,
       PD_WARM_EXTRAPOLATE = 4, PD_WARM_LEARNED_EXTRAP = 5 };
pd_status pd_set_warm_start(pd_sim* sim, int mode, pd_net* net);

/* Kinetic-energy histogram (eV) of one species, computed from raw particle
 * arrays in device memory, with no allocation of any kind.  The paper has no
 * counterpart: this is a service for callers that hold particles in their own
 * device buffers and cannot allocate device memory (the memory belongs to
 * another allocator or budget, or an allocation would synchronise the device
 * at a bad moment).  Inputs: n slots of key (species << 24 | cell, dead slots
 * 0xFFFFFFFF) and vz, vr, vt (m/s), all device pointers; out: nbins host
 * counters for [e_lo_eV, e_hi_eV), written before the call returns (the call
 * synchronises `cuda_stream`).  Bins are those of pd_get_energy_spectrum.
 * Scratch: one histogram of PD_SPECTRUM_STATIC_MAX_BINS counters in the
 * library's own device memory, which every GPU that loads the library keeps
 * until the process exits.  nbins above that maximum is rejected with
 * PD_ERR_ARG (pd_spectrum_static_max_bins() returns the maximum).  The
 * scratch belongs to the current device: `cuda_stream` must be a stream of
 * that device, else PD_ERR_ARG.  The first call on a device looks up the
 * scratch's device address and keeps it for the life of the process (it does
 * not survive a cudaDeviceReset).  The call synchronises `cuda_stream` (it
 * copies the histogram to the host before it returns), so it must not be
 * issued while any stream is being captured into a CUDA graph.  All calls
 * share the one histogram, which is cleared at the start of each call: calls
 * whose work overlaps on the GPU (other streams, other threads) race and give
 * wrong counts. */
#define PD_SPECTRUM_STATIC_MAX_BINS 4096
pd_status pd_energy_spectrum_static(const uint32_t* key, const float* vz, const float* vr, const float* vt,
                                    int64_t n, int species, double e_lo_eV, double e_hi_eV, int nbins,
                                    void* cuda_stream, uint64_t* out);
int pd_spectrum_static_max_bins(void);

#ifdef __cplusplus
}
#endif
#endif /* PD_H */
