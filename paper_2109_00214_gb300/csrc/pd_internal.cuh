// pd_internal.cuh -- device-side definitions shared by the library's kernels.
//
// Particle store (structure of arrays, one slot per super-particle):
//   key  u32  (species << 24) | cell, cell = iz * nr + ir; PD_DEAD for a free slot
//   pz, pr    f32 offset inside the cell, in [0, 1)
//   vz, vr, vt f32 velocity (m/s)
//   id   u32  particle id (ascending id = canonical order inside a cell)
// 28 bytes per particle.  Slots are grouped in bins, one per (species,
// cell), bin = species * cells + cell.  Heavy bins come first: heavy bin b
// owns slots [off[b], off[b+1]) and its live particles fill the first cnt[b]
// of them; the rest is slack (DEAD keys).  The electron bins follow, packed
// (rebuilt every step), from off[nbins] on; then the tail: particles created
// since the last sort (injected, spawned, sputtered, loaded).  A second copy
// (B) is scratch for the collisions and the target of a re-layout; a third
// (M) holds this step's movers at their slots' indices.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pd {

constexpr uint32_t DEAD = 0xFFFFFFFFu;
constexpr int NSP = 7;              // species codes; bins exist for the first KParams::nsp
constexpr int NCH = 9;
constexpr int SP_E = 0, SP_CU = 1, SP_CUP = 2, SP_CU2_SW = 3, SP_CU2_DI = 4, SP_CU3 = 5, SP_CU4 = 6;
// electron-impact channels, the heavy pairs of heavy steps (charge exchange
// Cu+ + Cu, elastic Cu + Cu; with heavy_coll), then the step-wise
// ionizations Cu2+ -> Cu3+ and Cu3+ -> Cu4+ (with charge_max 3 and 4)
constexpr int CH_EL = 0, CH_EXC = 1, CH_SI = 2, CH_DI = 3, CH_SW = 4, CH_CX = 5, CH_NN = 6, CH_S3 = 7, CH_S4 = 8;
// pair classes in the order a cell applies them: electron classes (e, Cu),
// (e, Cu+), (e, Cu2+ SW), (e, Cu2+ DI), (e, Cu3+), then the heavy pairs
// (Cu, Cu+) and (Cu, Cu)
constexpr int NCLS = 7, NECLS = 5;

// cross-section grid: 64 points per octave from 2^-10 eV over 25 octaves
constexpr int XS_EMIN_EXP = -10;
constexpr int XS_OCT = 25;
constexpr int XS_SUB = 64;
constexpr int XS_N = XS_OCT * XS_SUB + 1;

// sticky device error bits
constexpr uint32_t ERR_CAPACITY = 1u, ERR_TIMEOUT = 2u, ERR_NONFINITE = 4u, ERR_IDS = 8u, ERR_BOUNDS = 16u;

// counter slots (see PD_NCOUNTERS in pd.h)
constexpr int C_EV = 0, C_NULL = 5, C_CONSUMED = 6, C_THR = 7, C_VIOL = 8, C_ISOFB = 9, C_CAND = 10,
              C_EMIT_E = 11, C_EMIT_CU = 12, C_ABS = 13, C_EV_CX = 34, C_EV_NN = 35, C_EV_S3 = 36, C_EV_S4 = 37,
              C_COUL_EE = 38, C_COUL_EI = 39, C_SPUT_C = 40, C_SPUT_A = 41, C_COUL_II = 42, NCOUNTERS = 43;
// counter of the events of channel ch (channels 5-8 follow the absorption block)
__host__ __device__ constexpr int c_event(int ch) { return ch < CH_CX ? C_EV + ch : C_EV_CX + (ch - CH_CX); }

// Device-resident scalars shared by all runs of a simulation.
struct DevState {
    unsigned long long n_slots;      // slots of buffer A in use (live + dead)
    unsigned int n_heavy;            // cells with collision candidates this step: heavy ones (long
    unsigned int n_light;            // id lists or many candidates) and the others
    unsigned int error;              // ERR_* bits
    unsigned int load_bad;           // set by a device load that met an out-of-range particle
    unsigned int step;               // electron step index (Philox counter word), advanced by finalize
    unsigned int n_mid, n_big;       // id lists queued for the two rank-table kernels this step
    unsigned int collide_next;       // next active cell for k_collide's warps
    unsigned int n_sput;             // ion impacts recorded by the push for sputtering
    unsigned int relayout;           // a bin overflowed its slots this step: re-lay the bins out
    unsigned int since;              // steps since the last re-layout
    unsigned int n_bigc;             // long bins queued for the warp compaction this step
    unsigned int n_relayout;         // new layouts of the bins so far
    unsigned int sort_fault;         // which consistency check of the sort failed (bits), 0 if none
    unsigned int n_ovf;              // heavy bins that outgrew their slots this step
    unsigned long long n_live;       // heavy particles in bins (after this step's insertions)
    unsigned long long tail_base;    // first slot of the tail (after the electron bins)
    unsigned long long e_base;       // first slot of the electron bins (after the heavy bins' slots)
    unsigned long long e_from;       // the electron bins' first slot when this step's push ran
    unsigned long long n_e;          // electrons in bins
    unsigned long long sum_cnt;      // re-layout: particles over all bins, and the sums that size the
    double sum_s1, sum_s2;           // slack horizon (random-walk and drift terms)
    unsigned long long sp_cnt[NSP];  // re-layout: particles and bin traffic (movers in + out since
    unsigned long long sp_act[NSP];  // the last layout) of each species
};



// One ion impact on an electrode that sputters n atoms (recorded by the push,
// emitted by k_sputter in the order of the ions' ids).
struct SputRec {
    uint32_t id;                     // the ion's id
    uint32_t meta;                   // run << 1 | electrode (0 cathode, 1 anode)
    uint32_t ir;                     // radial cell of the impact (local)
    float pr;                        // radial offset of the impact in the cell
    uint32_t n;                      // atoms sputtered
};

// Device-resident scalars of one run (an ensemble holds several runs).
struct RunState {
    unsigned long long ctr[NCOUNTERS];
    double absorbed_energy[3];
    double charge_cathode;           // C through the cathode
    double anode_charge_step;        // C arriving at the anode this step
    double V;                        // anode voltage
    double I_gap;                    // last step's gap current
    double relres;                   // last Poisson relative residual
    double cycles;                   // last Poisson cycles
    double relres_max;               // largest final residual of the solves since it was last cleared
    double relres0;                  // last Poisson relative residual at the start of the solve
    unsigned int id_next;            // next particle id of the run
    unsigned int pad0;
};

// Per-run constants.  The runs' cells and nodes are laid end to end in one
// global index space: global cell = cell_base + iz * nr + ir.
struct RunInfo {
    int nz, nr, nzn, nrn;            // cells and nodes along z and r
    float inv_nr;                    // 1 / nr (cell decoding estimate)
    uint32_t cell_base, node_base, ncell;
    uint32_t seed, run;              // Philox key of the run
    uint32_t ck_base;                // c_k(j) of the run at ck[ck_base + k * nr + j]
    uint32_t row_base;               // W dt_coll / V_cell(j) of the run at cw[row_base + j]
    float qmdt[NSP];                 // z e / m * dt_s
    float dtz[NSP], dtr[NSP];        // dt_s / dz, dt_s / dr
    double weight;
};

// Collision constants (float; see the host's derivation).
struct CollConsts {
    float kmr;                       // eps[eV] = g^2 * kmr (electron-heavy pairs)
    float kmr_h;                     // the same for heavy pairs (m_r = M / 2)
    float a_e, a_t;                  // m_r / m_e, m_r / M
    float kth[NCH];                  // 2 E_th e / m_r
    float sgmax[NCLS];               // NTC majorants of the pair classes, in class order
    double kc[21];                   // Coulomb (q_a q_b)^2 lnL / (8 pi eps0^2 m_ab^2) of classes 0-20
    int di_split_mode;
};

struct Particles {
    uint32_t* key;
    float *pz, *pr, *vz, *vr, *vt;
    uint32_t* id;
};

// Launch-wide parameters passed by value to the kernels.
struct KParams {
    int geom;                        // 0 r-z, 1 periodic
    int nruns;
    uint32_t ncell;                  // cells of all runs
    uint32_t step;
    int heavy_step;
    int heavy_coll;                  // heavy pair classes on heavy steps
    int charge_max;                  // highest ion charge (2, 3 or 4): step-wise classes on
    int nsp;                         // species with bins: 5, or 7 with charge_max >= 3
    int coulomb;                     // Coulomb pair collisions after the DSMC classes
    uint32_t cw_heavy;               // heavy-step rows of cw follow the electron-step rows at this offset
    int sputter;                     // ions absorbed at the electrodes sputter atoms
    float sput_vth;                  // sqrt(k T_sputter / M)
    const float* xsE;                // the table grid (eV)
    const float* ytab;               // sputtering yield on the grid
    SputRec* squeue;                 // this step's impacts, at most squeue_cap
    uint32_t squeue_cap;
    int field_on;                    // gather E in the push
    unsigned long long capacity;     // physical slots of the particle arrays
    unsigned long long user_capacity;  // particles (live and reserved for spawns) the configuration allows
    double masses[NSP];
    RunInfo run0;                    // runs[0] by value (the one run of a single simulation)
    const RunInfo* runs;             // [nruns]
    const uint16_t* cell_run;        // run of each global cell (nruns > 1)
    RunState* rs;                    // [nruns]
};

constexpr int MAX_RUNS_SMEM = 128;   // kernels stage up to this many RunInfo in shared memory

// ---------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 S-box with
// multipliers 0xD2511F53, 0xCD9E8D57 and key increments 0x9E3779B9,
// 0xBB67AE85.
// ---------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Draw stream keyed by (subject, step, stream id); block counter in word 3.
struct Stream {
    uint4 ctr;
    uint2 key;
    uint4 buf;
    int used;
    __device__ __forceinline__ Stream(uint32_t subject, uint32_t step, uint32_t sid, uint32_t seed, uint32_t run)
        : ctr(make_uint4(subject, step, sid, 0u)), key(make_uint2(seed, run)), buf(make_uint4(0, 0, 0, 0)), used(4) {}
    __device__ __forceinline__ uint32_t next() {
        if (used == 4) {
            buf = philox4x32_10(ctr, key);
            ctr.w += 1u;
            used = 0;
        }
        const uint32_t v = used == 0 ? buf.x : used == 1 ? buf.y : used == 2 ? buf.z : buf.w;
        ++used;
        return v;
    }
    // uniform on [0, 1) from the top 24 bits
    __device__ __forceinline__ float u01() { return __fmul_rn((float)(next() >> 8), 5.9604644775390625e-08f); }
    // uniform integer in [0, n)
    __device__ __forceinline__ uint32_t pick(uint32_t n) { return (uint32_t)(((unsigned long long)next() * n) >> 32); }
};

__host__ __device__ constexpr uint32_t sid_cand(int k, uint32_t m) { return ((uint32_t)k << 28) | m; }
constexpr uint32_t SID_NCAND = 0xE0000000u;
// Coulomb classes 0 (e-e), 1-5 (e with Cu+, Cu2+ SW, Cu2+ DI, Cu3+, Cu4+) and
// 6-20 (ion pairs): pair k < 2^24 of class c (a range no other stream id
// uses), and the permutation keys of class c (SID_COUL_PERM | c)
__host__ __device__ constexpr uint32_t sid_coul(int c, uint32_t k) { return ((0x70u + (uint32_t)c) << 24) | k; }
constexpr uint32_t SID_COUL_PERM = 0xE1000000u;
constexpr uint32_t SID_INJ_COUNT = 0xD0000000u;
__host__ __device__ constexpr uint32_t sid_inj_e(uint32_t p) { return 0xD1000000u | p; }
__host__ __device__ constexpr uint32_t sid_inj_cu(uint32_t p) { return 0xD2000000u | p; }
// sputtering: an impact's count, and its j-th atom (subject: the ion's id)
constexpr uint32_t SID_SPUT = 0xD3000000u;
__host__ __device__ constexpr uint32_t sid_sput_atom(uint32_t j) { return 0xD4000000u | j; }

// Key layout: bits 0-23 cell, 24-26 species, 27-29 species before a
// conversion in this step's collisions, 31 "converted" flag (the sort needs
// the bin a particle was sorted under).  DEAD (all ones) is never a valid key.
constexpr uint32_t KEY_FLAG = 0x80000000u;
__device__ __forceinline__ uint32_t key_species(uint32_t key) { return (key >> 24) & 7u; }
__device__ __forceinline__ uint32_t key_sorted_species(uint32_t key) {
    return (key & KEY_FLAG) ? ((key >> 27) & 7u) : ((key >> 24) & 7u);
}
__device__ __forceinline__ uint32_t key_cell(uint32_t key) { return key & 0xFFFFFFu; }
__device__ __forceinline__ uint32_t make_key(uint32_t sp, uint32_t cell) { return (sp << 24) | cell; }
__device__ __forceinline__ uint32_t converted_key(uint32_t new_sp, uint32_t old_sp, uint32_t cell) {
    return KEY_FLAG | (old_sp << 27) | (new_sp << 24) | cell;
}

// particle masses (CODATA 2018; every Cu charge state has the atom's mass)
constexpr double MASS_E = 9.1093837015e-31;
constexpr double AMU_KG = 1.66053906660e-27;
constexpr double MASS_CU = 63.546 * AMU_KG;
__host__ __device__ constexpr double species_mass_kg(int sp) { return sp == SP_E ? MASS_E : MASS_CU; }

// charge number: e -1, Cu 0, Cu+ 1, Cu2+ (both labels) 2, Cu3+ 3, Cu4+ 4
// (charge + 1 of species sp in nibble sp)
__host__ __device__ __forceinline__ int charge_of(int sp) { return (int)((0x5433210u >> (4 * sp)) & 15u) - 1; }

// global node index of local node (i, j) of a run; periodic wrap in the
// Cartesian mode
__device__ __forceinline__ uint32_t node_of(const RunInfo& R, int geom, int i, int j) {
    if (geom != 0) {
        if (i >= R.nz) i -= R.nz;
        if (j >= R.nr) j -= R.nr;
        return R.node_base + (uint32_t)i * (uint32_t)R.nr + (uint32_t)j;
    }
    return R.node_base + (uint32_t)i * (uint32_t)R.nrn + (uint32_t)j;
}

// run of a global cell
__device__ __forceinline__ int run_of(const KParams& P, uint32_t gcell) {
    return P.nruns == 1 ? 0 : (int)P.cell_run[gcell];
}

__device__ __forceinline__ void set_error(DevState* st, uint32_t bits) { atomicOr(&st->error, bits); }

// sigma(eps): linear interpolation on the grid E_k = 2^e (1 + j/64); the
// bracketing index comes from the exponent and top six mantissa bits of eps.
__device__ __forceinline__ float xs_lookup(const float* __restrict__ E, const float* __restrict__ s, float eps) {
    if (!(eps < E[XS_N - 1])) return 0.0f;
    int k;
    if (eps < E[0]) {
        k = 0;
        eps = E[0];
    } else {
        const uint32_t b = __float_as_uint(eps);
        k = ((int)(b >> 23) - 127 - XS_EMIN_EXP) * XS_SUB + (int)((b >> 17) & 63u);
    }
    const float t = (eps - E[k]) / (E[k + 1] - E[k]);
    return s[k] + t * (s[k + 1] - s[k]);
}


}  // namespace pd
