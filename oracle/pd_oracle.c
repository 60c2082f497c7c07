/*
 * pd_oracle.c -- plain, slow CPU oracle of the 2D3V PIC-DSMC time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA library: its Philox generator, cross-section lookup, push, deposit,
 * collision kinematics and field solve are written here from the paper and
 * from the published definitions they name.
 *
 * One source, two builds:
 *   -DOR_DOUBLE   every particle quantity in double (physics checks);
 *   (default)     float "mirror" mode: the same float operations in the same
 *                 order as the method's FP32 state, so that event counts,
 *                 labels and fixed-point charge can be compared bit for bit.
 * Build with -ffp-contract=off so that no multiply-add is fused.
 *
 * Paper: W. Yang et al., "The role of double ionization on the generation of
 * doubly charged ions in copper vacuum arcs" (arXiv:2109.00214).
 *   Sec. 2.1 Eq. (1)-(10): PIC-DSMC, pair collision probability, momentum
 *            and energy conserving post-collision velocities, CIC weighting,
 *            Verboncoeur volumes.
 *   Sec. 2.2 Eq. (11)-(20): four-stage double-ionization scheme with the
 *            velocity rectangle split.
 *   Sec. 2.3: r-z geometry, 1 fs / 10 fs steps, W = 100, RC circuit, FN tip,
 *            3 % neutral flux, channel-labelled Cu2+.
 *   Sec. 3.1 Eq. (21): ionization degree and mean charge.
 *
 * Parity pins (what fixes each part independently of this file) are listed
 * in the tests; the cross-section data of the paper (its Fig. 1, refs.
 * [28-30]) is not available, so the tables are inputs.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* The OpenMP build (OR_OMP) runs the particle loops and the cells'
 * collisions on all host cores.  It is deterministic and gives the serial
 * build's particles, counts and charge: deposits are integer, a cell's
 * collisions are ordered and touch only its particles, spawns take the
 * slots their ids reserve and are compacted in order; only the FP64 ledger
 * sums (energies, the gap current) are added in another order. */
#ifdef OR_OMP
#include <omp.h>
#define OR_ATOMIC _Pragma("omp atomic")
#else
#define OR_ATOMIC
#endif

#ifdef OR_DOUBLE
typedef double real;
#define R_(x) ((double)(x))
#define OR_SQRT sqrt
#define OR_FLOOR floor
#define OR_NEXTAFTER nextafter
#else
typedef float real;
#define R_(x) ((float)(x))
#define OR_SQRT sqrtf
#define OR_FLOOR floorf
#define OR_NEXTAFTER nextafterf
#endif

/* ------------------------------------------------------------------ */
/* physical constants (CODATA 2018)                                    */
/* ------------------------------------------------------------------ */
static const double QE = 1.602176634e-19;
static const double ME = 9.1093837015e-31;
static const double AMU = 1.66053906660e-27;
static const double EPS0 = 8.8541878128e-12;
static const double KB = 1.380649e-23;
#define M_CU (63.546 * AMU)
static const double PI = 3.14159265358979323846;

/* Cu3+ and Cu4+ are the higher charge states Sec. 2.3 tracks; they exist   */
/* only with charge_max 3 or 4                                             */
enum { SP_E = 0, SP_CU = 1, SP_CUP = 2, SP_CU2_SW = 3, SP_CU2_DI = 4, SP_CU3 = 5, SP_CU4 = 6, NSP = 7 };
/* channels 5 and 6 are the heavy-particle collisions the paper lists     */
/* besides ionization (Sec. 2.3): charge exchange Cu+ + Cu and elastic    */
/* Cu + Cu; off unless heavy_coll is set.  Channels 7 and 8 are the       */
/* step-wise ionizations Cu2+ -> Cu3+ and Cu3+ -> Cu4+ (Sec. 2.3), on      */
/* with charge_max >= 3 and 4                                             */
enum { CH_EL = 0, CH_EXC = 1, CH_SI = 2, CH_DI = 3, CH_SW = 4, CH_CX = 5, CH_NN = 6, CH_S3 = 7, CH_S4 = 8,
       NCH = 9 };
static const int ZQ[NSP] = {-1, 0, 1, 2, 2, 3, 4};

/* cross-section grid (must be the grid the inputs are tabulated on) */
#define XS_EMIN_EXP (-10)
#define XS_OCT 25
#define XS_SUB 64
#define XS_N (XS_OCT * XS_SUB + 1)

/* ------------------------------------------------------------------ */
/* configuration (filled by oracle/__init__.py)                       */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t geom;          /* 0 = r-z with electrodes, 1 = Cartesian periodic */
    int32_t nz, nr;
    double dz, dr, depth, dt;
    int32_t heavy_subcycle;
    double weight;
    uint32_t seed, run;
    int32_t field_mode;    /* 0 none, 1 Poisson each step, 2 external fixed field */
    int32_t inject_on, di_on, di_split_mode;
    double coll_dt_scale;
    double V0, R_ohm, C_farad;
    double beta, tip_radius, work_function, neutral_ratio, neutral_T;
    double poisson_tol;
    int64_t capacity;
    int32_t heavy_coll;    /* heavy-particle pair classes (charge exchange, Cu-Cu elastic) on */
    int32_t charge_max;    /* highest ion charge: 2 (Cu2+), 3 (+ Cu2+ -> Cu3+), 4 (+ Cu3+ -> Cu4+) */
    int32_t coulomb;       /* Coulomb collisions e-e and e-ion (binary collision model) on */
    double coulomb_lnl;    /* Coulomb logarithm */
    int32_t sputter;       /* ion-impact sputtering at the electrodes on */
    double sputter_T;      /* temperature (K) of the sputtered atoms' effusive flux */
} or_cfg;

typedef struct {
    or_cfg c;
    int64_t n, cap;
    uint8_t *sp;
    int32_t *iz, *ir;
    real *pz, *pr, *vz, *vr, *vt;
    uint32_t *id;
    uint32_t id_next;
    uint32_t step;
    /* nodes */
    int nzn, nrn;          /* node counts */
    int64_t *rho_e, *rho_h;
    double *phi;
    real *Ez, *Er;
    double V;              /* anode voltage */
    double I_gap;          /* last step's gap current */
    /* cross sections: sigma[ch][k] on E_k */
    float xsE[XS_N];
    real xs[NCH][XS_N];
    double eth[NCH];
    real sgmax[7];
    /* counters */
    uint64_t events[NCH], nulls, consumed, thr_rej, ratio_viol, iso_fallback, cand_total;
    uint64_t coul_ee, coul_ei, coul_ii;   /* Coulomb pair collisions applied: e-e, e-ion, ion-ion */
    uint64_t sput[2];            /* atoms sputtered from the cathode, the anode */
    real ytab[XS_N];             /* sputtering yield Y(E) on the cross-section grid */
    struct sput_rec* srec;       /* this step's ion impacts on the electrodes */
    int64_t nsrec, srec_cap;
    uint64_t absorbed[3][NSP];   /* cathode, anode, outer wall */
    double absorbed_energy[3];   /* J (physical, includes W) */
    uint64_t emitted_e, emitted_cu;
    double charge_cathode;       /* C, net charge through the cathode */
    float ray[1024];             /* Rayleigh inverse CDF in units of sigma */
    int poisson_iters;
    double poisson_relres;
    /* collisions of cells in parallel: spawns go to the slot their id
     * reserves, spawn_base + (id - spawn_id0) */
    int spawn_mode;
    int64_t spawn_base;
    uint32_t spawn_id0;
} or_sim;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:  */
/* as easy as 1, 2, 3", SC'11): ten rounds of the 4x32 S-box on a       */
/* 128-bit counter with a 64-bit key bumped by the Weyl constants.      */
/* ------------------------------------------------------------------ */
static void philox10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void or_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox10(ctr, key, out); }

/* A draw stream: counter (subject, step, stream id, block), four words per
 * block, consumed in order. */
typedef struct {
    uint32_t ctr[4], key[2], buf[4];
    int used;
} stream_t;

static void stream_init(stream_t* s, const or_sim* S, uint32_t subject, uint32_t step, uint32_t sid) {
    s->ctr[0] = subject; s->ctr[1] = step; s->ctr[2] = sid; s->ctr[3] = 0;
    s->key[0] = S->c.seed; s->key[1] = S->c.run;
    s->used = 4;
}
static uint32_t next_u32(stream_t* s) {
    if (s->used == 4) {
        philox10(s->ctr, s->key, s->buf);
        s->ctr[3] += 1;
        s->used = 0;
    }
    return s->buf[s->used++];
}
/* uniform on [0, 1): float from the top 24 bits, double from 53 bits of two words */
static real u01(stream_t* s) {
#ifdef OR_DOUBLE
    uint32_t a = next_u32(s), b = next_u32(s);
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
#else
    return (float)(next_u32(s) >> 8) * (1.0f / 16777216.0f);
#endif
}
/* uniform integer in [0, n) by the 32x32 -> 64 multiply-high */
static uint32_t pick(stream_t* s, uint32_t n) { return (uint32_t)(((uint64_t)next_u32(s) * n) >> 32); }

/* stream ids (third counter word) */
#define SID_CAND(k, m) (((uint32_t)(k) << 28) | (uint32_t)(m))
#define SID_NCAND 0xE0000000u
/* Coulomb classes 0 (e-e), 1-5 (e with Cu+, Cu2+ SW, Cu2+ DI, Cu3+, Cu4+)
 * and 6-20 (ion pairs): pair k < 2^24 of class c, and the permutation keys
 * of class c (a range no other stream id uses) */
#define SID_COUL(c, k) (((0x70u + (uint32_t)(c)) << 24) | (uint32_t)(k))
#define SID_COUL_PERM(c) (0xE1000000u | (uint32_t)(c))
#define SID_INJ_COUNT 0xD0000000u
#define SID_INJ_E(p) (0xD1000000u | (uint32_t)(p))
#define SID_INJ_CU(p) (0xD2000000u | (uint32_t)(p))
/* sputtering: the count of an ion impact, the j-th sputtered atom (subject: the ion's id) */
#define SID_SPUT 0xD3000000u
#define SID_SPUT_ATOM(j) (0xD4000000u | (uint32_t)(j))

/* ------------------------------------------------------------------ */
/* geometry                                                             */
/* ------------------------------------------------------------------ */
/* cell volume: r-z annulus pi((j+1)^2 - j^2) dr^2 dz, else dz dr depth */
static double cell_volume(const or_sim* S, int j) {
    if (S->c.geom == 0) return PI * (double)(2 * j + 1) * S->c.dr * S->c.dr * S->c.dz;
    return S->c.dz * S->c.dr * S->c.depth;
}
/* Node volume for charge density, Eq. (9) with Verboncoeur's volumes [24]:
 * V_j = 2 pi dz_eff * integral of the linear hat S_j(r) r dr, i.e. axis
 * pi dz dr^2 / 3, interior 2 pi dz dr^2 j, outer 2 pi dz dr^2 (N/2 - 1/6);
 * electrode nodes have half the axial extent. */
static double node_volume(const or_sim* S, int i, int j) {
    if (S->c.geom != 0) return S->c.dz * S->c.dr * S->c.depth;
    double dz = S->c.dz, dr = S->c.dr;
    int N = S->c.nr;
    double v;
    if (j == 0) v = PI * dz * dr * dr / 3.0;
    else if (j == N) v = 2.0 * PI * dz * dr * dr * ((double)N / 2.0 - 1.0 / 6.0);
    else v = 2.0 * PI * dz * dr * dr * (double)j;
    if (i == 0 || i == S->c.nz) v *= 0.5;
    return v;
}
static int64_t node_index(const or_sim* S, int i, int j) {
    if (S->c.geom != 0) {
        i %= S->c.nz; j %= S->c.nr;
        return (int64_t)i * S->c.nr + j;
    }
    return (int64_t)i * (S->c.nr + 1) + j;
}
static double species_mass(int s) { return s == SP_E ? ME : M_CU; }

/* ------------------------------------------------------------------ */
/* cross sections: piecewise-linear in E on the grid                     */
/* ------------------------------------------------------------------ */
static void xs_build_grid(or_sim* S) {
    for (int k = 0; k < XS_N; ++k) {
        int e = XS_EMIN_EXP + k / XS_SUB, j = k % XS_SUB;
        S->xsE[k] = (float)ldexp(1.0 + (double)j / XS_SUB, e);
    }
}
/* sigma_c(eps) by linear interpolation between the bracketing grid points;
 * below the first point the first value, at or above the last point zero. */
/* linear interpolation of a table on the cross-section grid, 0 at or above
 * the grid's end, the first value below its start */
static real tab_lookup(const or_sim* S, const real* tab, real eps) {
    if (!(eps < (real)S->xsE[XS_N - 1])) return R_(0);
    int k;
    if (eps < (real)S->xsE[0]) {
        k = 0; eps = (real)S->xsE[0];
    } else {
        int lo = 0, hi = XS_N - 1;       /* xsE[lo] <= eps < xsE[hi] */
        while (hi - lo > 1) {
            int mid = (lo + hi) / 2;
            if ((real)S->xsE[mid] <= eps) lo = mid; else hi = mid;
        }
        k = lo;
    }
    real t = (eps - (real)S->xsE[k]) / ((real)S->xsE[k + 1] - (real)S->xsE[k]);
    return tab[k] + t * (tab[k + 1] - tab[k]);
}
static real xs_lookup(const or_sim* S, int ch, real eps) { return tab_lookup(S, S->xs[ch], eps); }

/* pair classes, in the order a cell applies them: the electron classes
 * (e, Cu), (e, Cu+), (e, Cu2+ SW), (e, Cu2+ DI), (e, Cu3+) (the last three
 * with charge_max >= 3, 3, 4), then, on heavy steps with heavy_coll,
 * (Cu, Cu+) charge exchange and (Cu, Cu) elastic */
#define NCLS 7
#define NECLS 5
static const int CLASS_CH0[NCLS] = {CH_EL, CH_SW, CH_S3, CH_S3, CH_S4, CH_CX, CH_NN};
static const int CLASS_NCH[NCLS] = {4, 1, 1, 1, 1, 1, 1};
static const int CLASS_TARGET[NCLS] = {SP_CU, SP_CUP, SP_CU2_SW, SP_CU2_DI, SP_CU3, SP_CUP, SP_CU};
/* highest ion charge a class needs */
static const int CLASS_QMAX[NCLS] = {2, 2, 3, 3, 4, 2, 2};

static double mr_class(void) { return ME * M_CU / (ME + M_CU); }
static real kmr(void) { return R_(0.5 * mr_class() / QE); } /* eps[eV] = g^2 * kmr */
/* heavy pairs: equal masses, m_r = M/2 */
static real kmr_heavy(void) { return R_(0.5 * (0.5 * M_CU) / QE); }

/* NTC majorant (sigma g)_max of one pair class: on each grid segment the
 * interpolant is at most the larger end value and g is largest at the upper
 * end, so max_k max(sT_k, sT_k+1) * g(E_k+1) bounds sigma_T(eps) g(eps); a
 * relative margin of 1e-6 covers float rounding. */
static void compute_sgmax(or_sim* S) {
    for (int k = 0; k < NCLS; ++k) {
        double kd = (double)(k < NECLS ? kmr() : kmr_heavy());
        double best = 0.0;
        real sT_prev = 0;
        for (int q = 0; q < XS_N; ++q) {
            real sT = 0;
            for (int c = 0; c < CLASS_NCH[k]; ++c) sT = sT + S->xs[CLASS_CH0[k] + c][q];
            if (q > 0) {
                real smax = sT > sT_prev ? sT : sT_prev;
                double g = sqrt((double)S->xsE[q] / kd);
                double cand = (double)smax * g;
                if (cand > best) best = cand;
            }
            sT_prev = sT;
        }
        best *= 1.0 + 1e-6;
        real f = R_(best);
        if ((double)f < best) f = OR_NEXTAFTER(f, INFINITY);
        S->sgmax[k] = f;
    }
}

/* ------------------------------------------------------------------ */
/* lifecycle                                                            */
/* ------------------------------------------------------------------ */
or_sim* or_create(const or_cfg* c) {
    or_sim* S = (or_sim*)calloc(1, sizeof(or_sim));
    S->c = *c;
    S->cap = c->capacity;
    S->sp = (uint8_t*)malloc(S->cap);
    S->iz = (int32_t*)malloc(S->cap * 4);
    S->ir = (int32_t*)malloc(S->cap * 4);
    S->pz = (real*)malloc(S->cap * sizeof(real));
    S->pr = (real*)malloc(S->cap * sizeof(real));
    S->vz = (real*)malloc(S->cap * sizeof(real));
    S->vr = (real*)malloc(S->cap * sizeof(real));
    S->vt = (real*)malloc(S->cap * sizeof(real));
    S->id = (uint32_t*)malloc(S->cap * 4);
    if (c->geom == 0) { S->nzn = c->nz + 1; S->nrn = c->nr + 1; }
    else { S->nzn = c->nz; S->nrn = c->nr; }
    int64_t nn = (int64_t)S->nzn * S->nrn;
    S->rho_e = (int64_t*)calloc(nn, 8);
    S->rho_h = (int64_t*)calloc(nn, 8);
    S->phi = (double*)calloc(nn, 8);
    S->Ez = (real*)calloc(nn, sizeof(real));
    S->Er = (real*)calloc(nn, sizeof(real));
    S->V = c->V0;
    xs_build_grid(S);
    /* Rayleigh inverse CDF sqrt(-2 ln(1 - U)) at U = k/1024 (units of the
     * thermal speed), for the effusive neutral source. */
    for (int k = 0; k < 1024; ++k) S->ray[k] = (float)sqrt(-2.0 * log(1.0 - (double)k / 1024.0));
    return S;
}

void or_destroy(or_sim* S) {
    if (!S) return;
    free(S->sp); free(S->iz); free(S->ir); free(S->pz); free(S->pr);
    free(S->vz); free(S->vr); free(S->vt); free(S->id);
    free(S->rho_e); free(S->rho_h); free(S->phi); free(S->Ez); free(S->Er);
    free(S->srec);
    free(S);
}

/* Cross section of one channel, given as (E_eV, sigma_m2) pairs (ascending
 * E); resampled by linear interpolation onto the grid (identity when the
 * input already sits on the grid).  Zero below the threshold. */
/* sputtering yield Y(E) (sputtered atoms per ion, E the impact energy in eV),
 * resampled onto the cross-section grid like the cross sections */
int or_set_yield(or_sim* S, const double* E, const double* Y, int n) {
    if (n < 2) return 1;
    for (int k = 0; k < XS_N; ++k) {
        double e = (double)S->xsE[k], v;
        if (e <= E[0]) v = Y[0];
        else if (e >= E[n - 1]) v = Y[n - 1];
        else {
            int a = 0;
            while (E[a + 1] <= e) ++a;
            double t = (e - E[a]) / (E[a + 1] - E[a]);
            v = Y[a] + t * (Y[a + 1] - Y[a]);
        }
        S->ytab[k] = R_(v);
    }
    return 0;
}

int or_set_xs(or_sim* S, int ch, const double* E, const double* sig, int n, double threshold) {
    if (ch < 0 || ch >= NCH || n < 2) return 1;
    for (int k = 0; k < XS_N; ++k) {
        double e = (double)S->xsE[k], v;
        if (e <= E[0]) v = sig[0];
        else if (e >= E[n - 1]) v = sig[n - 1];
        else {
            int a = 0;
            while (E[a + 1] <= e) ++a;
            double t = (e - E[a]) / (E[a + 1] - E[a]);
            v = sig[a] + t * (sig[a + 1] - sig[a]);
        }
        if (e < threshold) v = 0.0;
        if (ch == CH_DI && !S->c.di_on) v = 0.0;
        S->xs[ch][k] = R_(v);
    }
    S->eth[ch] = threshold;
    compute_sgmax(S);
    return 0;
}

/* Append particles (cell-relative positions); ids follow in load order. */
int64_t or_load(or_sim* S, int64_t n, const uint8_t* sp, const int32_t* iz, const int32_t* ir,
                const double* pz, const double* pr, const double* vz, const double* vr, const double* vt) {
    if (S->n + n > S->cap) return -1;
    /* species codes beyond the configured highest charge are refused */
    for (int64_t q = 0; q < n; ++q)
        if (sp[q] >= NSP || ZQ[sp[q]] > S->c.charge_max) return -2;
    for (int64_t q = 0; q < n; ++q) {
        int64_t p = S->n + q;
        S->sp[p] = sp[q]; S->iz[p] = iz[q]; S->ir[p] = ir[q];
        S->pz[p] = R_(pz[q]); S->pr[p] = R_(pr[q]);
        S->vz[p] = R_(vz[q]); S->vr[p] = R_(vr[q]); S->vt[p] = R_(vt[q]);
        S->id[p] = S->id_next++;
    }
    S->n += n;
    return S->n;
}

void or_set_field(or_sim* S, const double* Ez, const double* Er) {
    int64_t nn = (int64_t)S->nzn * S->nrn;
    for (int64_t k = 0; k < nn; ++k) { S->Ez[k] = R_(Ez[k]); S->Er[k] = R_(Er[k]); }
}

/* ------------------------------------------------------------------ */
/* push: Newton's law for each super-particle (Sec. 2.1), leapfrog with    */
/* v at half steps; r-z motion done in the local Cartesian frame and       */
/* rotated back.  Field gathered with the CIC weights of Eq. (10).         */
/* Returns 0 if the particle stays, 1 + electrode if it leaves.           */
/* ------------------------------------------------------------------ */
static const real ONE_MINUS_ULP =
#ifdef OR_DOUBLE
    0x1.fffffffffffffp-1;
#else
    0x1.fffffep-1f;
#endif

static int push_one(or_sim* S, int64_t p, real qmdt, real dtz, real dtr) {
    real vz = S->vz[p], vr = S->vr[p], vt = S->vt[p];
    real pz = S->pz[p], pr = S->pr[p];
    int iz = S->iz[p], ir = S->ir[p];
    if (S->c.field_mode != 0) {
        real gz = R_(1) - pz, gr = R_(1) - pr;
        int64_t n00 = node_index(S, iz, ir), n10 = node_index(S, iz + 1, ir);
        int64_t n01 = node_index(S, iz, ir + 1), n11 = node_index(S, iz + 1, ir + 1);
        real w00 = gz * gr, w10 = pz * gr, w01 = gz * pr, w11 = pz * pr;
        real Ez = ((w00 * S->Ez[n00] + w10 * S->Ez[n10]) + w01 * S->Ez[n01]) + w11 * S->Ez[n11];
        real Er = ((w00 * S->Er[n00] + w10 * S->Er[n10]) + w01 * S->Er[n01]) + w11 * S->Er[n11];
        vz = vz + qmdt * Ez;
        vr = vr + qmdt * Er;
    }
    /* axial move, in cell units */
    real z = pz + vz * dtz;
    real fz = OR_FLOOR(z);
    int niz = iz + (int)fz;
    real npz = z - fz;
    if (npz >= R_(1)) npz = ONE_MINUS_ULP;
    int nir;
    real npr;
    if (S->c.geom == 0) {
        /* r-z: x = r + v_r dt, y = v_theta dt; r' = |(x, y)|; rotate (v_r, v_theta) */
        real x = ((real)ir + pr) + vr * dtr;
        real y = vt * dtr;
        real rr = OR_SQRT(x * x + y * y);
        real cth = R_(1), sth = R_(0);
        if (rr > R_(0)) { cth = x / rr; sth = y / rr; }
        real nvr = cth * vr + sth * vt;
        real nvt = cth * vt - sth * vr;
        vr = nvr; vt = nvt;
        real fr = OR_FLOOR(rr);
        nir = (int)fr;
        npr = rr - fr;
        if (npr >= R_(1)) npr = ONE_MINUS_ULP;
    } else {
        real r = pr + vr * dtr;
        real fr = OR_FLOOR(r);
        nir = ir + (int)fr;
        npr = r - fr;
        if (npr >= R_(1)) npr = ONE_MINUS_ULP;
    }
    S->vz[p] = vz; S->vr[p] = vr; S->vt[p] = vt;
    S->pz[p] = npz; S->pr[p] = npr;
    if (S->c.geom != 0) {
        int nz = S->c.nz, nr = S->c.nr;
        niz = ((niz % nz) + nz) % nz;
        nir = ((nir % nr) + nr) % nr;
        S->iz[p] = niz; S->ir[p] = nir;
        return 0;
    }
    S->iz[p] = niz; S->ir[p] = nir;
    if (niz < 0) return 1;           /* cathode z = 0 */
    if (niz >= S->c.nz) return 2;    /* anode z = L */
    if (nir >= S->c.nr) return 3;    /* outer wall r = R */
    return 0;
}

/* ------------------------------------------------------------------ */
/* deposit: Eq. (9)-(10) CIC in fixed point.  Per axis w = round-to-     */
/* nearest-even(f * 2^16) with f the cell-relative offset; the four       */
/* corner weights are products of (2^16 - w) and w and sum to 2^32.       */
/* ------------------------------------------------------------------ */
static void deposit_one(const or_sim* S, int64_t* rho, int iz, int ir, real pz, real pr, int64_t zq) {
    uint32_t wz = (uint32_t)nearbyint((double)(pz * R_(65536)));
    uint32_t wr = (uint32_t)nearbyint((double)(pr * R_(65536)));
    int64_t az = 65536 - (int64_t)wz, ar = 65536 - (int64_t)wr;
    OR_ATOMIC rho[node_index(S, iz, ir)] += zq * az * ar;
    OR_ATOMIC rho[node_index(S, iz + 1, ir)] += zq * (int64_t)wz * ar;
    OR_ATOMIC rho[node_index(S, iz, ir + 1)] += zq * az * (int64_t)wr;
    OR_ATOMIC rho[node_index(S, iz + 1, ir + 1)] += zq * (int64_t)wz * (int64_t)wr;
}

static void remove_particle(or_sim* S, int64_t p) {
    int64_t q = S->n - 1;
    S->sp[p] = S->sp[q]; S->iz[p] = S->iz[q]; S->ir[p] = S->ir[q];
    S->pz[p] = S->pz[q]; S->pr[p] = S->pr[q];
    S->vz[p] = S->vz[q]; S->vr[p] = S->vr[q]; S->vt[p] = S->vt[q];
    S->id[p] = S->id[q];
    S->n--;
}

static int64_t append_particle(or_sim* S, int sp, int iz, int ir, real pz, real pr,
                               real vz, real vr, real vt, uint32_t id) {
    if (S->n >= S->cap) return -1;
    int64_t p = S->n++;
    S->sp[p] = (uint8_t)sp; S->iz[p] = iz; S->ir[p] = ir;
    S->pz[p] = pz; S->pr[p] = pr; S->vz[p] = vz; S->vr[p] = vr; S->vt[p] = vt;
    S->id[p] = id;
    return p;
}

/* a particle made by a collision: appended, or (cells in parallel) put in
 * the slot its id reserves */
static int64_t spawn_particle(or_sim* S, int sp, int iz, int ir, real pz, real pr, real vz, real vr, real vt,
                              uint32_t id) {
    if (!S->spawn_mode) return append_particle(S, sp, iz, ir, pz, pr, vz, vr, vt, id);
    int64_t p = S->spawn_base + (int64_t)(id - S->spawn_id0);
    S->sp[p] = (uint8_t)sp; S->iz[p] = iz; S->ir[p] = ir;
    S->pz[p] = pz; S->pr[p] = pr; S->vz[p] = vz; S->vr[p] = vr; S->vt[p] = vt;
    S->id[p] = id;
    return p;
}

static double kinetic(const or_sim* S, int64_t p) {
    double v2 = (double)S->vz[p] * S->vz[p] + (double)S->vr[p] * S->vr[p] + (double)S->vt[p] * S->vt[p];
    return 0.5 * species_mass(S->sp[p]) * v2;
}

/* ------------------------------------------------------------------ */
/* Ion-impact sputtering (Sec. 2.3: energetic ions arriving at the        */
/* electrodes sputter neutrals into the domain, yield of Yamamura and     */
/* Tawara [32]; the yield is an input table here).  An ion super-particle */
/* of impact energy E absorbed at the cathode or the anode yields         */
/* floor(Y(E) + R) Cu super-particles of the same weight, emitted from the */
/* impact point (same r, on the electrode surface) into the gap with an    */
/* effusive flux at sputter_T: Rayleigh normal and transverse speeds,      */
/* uniform azimuth.  Impacts are taken in ascending ion id, so the new     */
/* atoms' ids do not depend on the order of the push.  An impact beyond    */
/* the outer radius (a corner crossing) sputters nothing.                 */
/* ------------------------------------------------------------------ */
typedef struct sput_rec { uint32_t id; int el; int ir; real pr; real Y; } sput_rec;

static int cmp_sput(const void* a, const void* b) {
    uint32_t x = ((const sput_rec*)a)->id, y = ((const sput_rec*)b)->id;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static void sputter_record(or_sim* S, int64_t p, int el) {
    if (S->ir[p] >= S->c.nr) return;
    if (S->nsrec == S->srec_cap) {
        S->srec_cap = S->srec_cap ? 2 * S->srec_cap : 1024;
        S->srec = (sput_rec*)realloc(S->srec, (size_t)S->srec_cap * sizeof(sput_rec));
    }
    sput_rec* r = &S->srec[S->nsrec++];
    r->id = S->id[p];
    r->el = el;
    r->ir = S->ir[p];
    r->pr = S->pr[p];
    r->Y = tab_lookup(S, S->ytab, R_(kinetic(S, p) / QE));
}

static real rayleigh(const or_sim* S, real U);
static void azimuth(or_sim* S, stream_t* st, real* c, real* s);

static int sputter_emit(or_sim* S) {
    if (S->nsrec > 1) qsort(S->srec, (size_t)S->nsrec, sizeof(sput_rec), cmp_sput);
    real vth = R_(sqrt(KB * S->c.sputter_T / M_CU));
    for (int64_t q = 0; q < S->nsrec; ++q) {
        const sput_rec* r = &S->srec[q];
        stream_t st;
        stream_init(&st, S, r->id, S->step, SID_SPUT);
        uint32_t n = (uint32_t)OR_FLOOR(r->Y + u01(&st));
        for (uint32_t j = 0; j < n; ++j) {
            stream_t sp;
            stream_init(&sp, S, r->id, S->step, SID_SPUT_ATOM(j));
            real U1 = u01(&sp), U2 = u01(&sp);
            real vn = vth * rayleigh(S, U1);
            real s = vth * rayleigh(S, U2);
            real cp, sn;
            azimuth(S, &sp, &cp, &sn);
            int iz = r->el == 0 ? 0 : S->c.nz - 1;
            real pz = r->el == 0 ? R_(0) : ONE_MINUS_ULP;
            if (append_particle(S, SP_CU, iz, r->ir, pz, r->pr, r->el == 0 ? vn : -vn, s * cp, s * sn,
                                S->id_next++) < 0)
                return 1;
            S->sput[r->el]++;
        }
    }
    S->nsrec = 0;
    return 0;
}

#ifdef OR_OMP
/* the push on all cores: every particle is pushed on its own; then, in index
 * order, the absorbed ones are tallied and the others kept (stable) */
static void push_all_par(or_sim* S, int heavy_step) {
    double dte = S->c.dt, dth = S->c.dt * S->c.heavy_subcycle;
    int64_t n = S->n;
    uint8_t* out = (uint8_t*)malloc(n > 0 ? (size_t)n : 1);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
        int s = S->sp[p];
        out[p] = 0;
        if (s != SP_E && !heavy_step) continue;
        double dts = (s == SP_E) ? dte : dth;
        real qmdt = R_((double)ZQ[s] * QE / species_mass(s) * dts);
        real dtz = R_(dts / S->c.dz), dtr = R_(dts / S->c.dr);
        out[p] = (uint8_t)push_one(S, p, qmdt, dtz, dtr);
    }
    double IgapQ = 0.0;
    int64_t w = 0;
    for (int64_t p = 0; p < n; ++p) {
        if (out[p]) {
            int s = S->sp[p], el = out[p] - 1;
            S->absorbed[el][s] += 1;
            S->absorbed_energy[el] += S->c.weight * kinetic(S, p);
            if (el == 1) IgapQ += -(double)ZQ[s] * QE * S->c.weight;
            if (el == 0) S->charge_cathode += (double)ZQ[s] * QE * S->c.weight;
            continue;
        }
        if (w != p) {
            S->sp[w] = S->sp[p]; S->iz[w] = S->iz[p]; S->ir[w] = S->ir[p];
            S->pz[w] = S->pz[p]; S->pr[w] = S->pr[p];
            S->vz[w] = S->vz[p]; S->vr[w] = S->vr[p]; S->vt[w] = S->vt[p];
            S->id[w] = S->id[p];
        }
        ++w;
    }
    S->n = w;
    S->I_gap = IgapQ / dte;
    free(out);
}
#endif

static void push_all(or_sim* S, int heavy_step) {
#ifdef OR_OMP
    if (!S->c.sputter) {       /* (the impact records of sputtering are kept in the serial order) */
        push_all_par(S, heavy_step);
        return;
    }
#endif
    double dte = S->c.dt, dth = S->c.dt * S->c.heavy_subcycle;
    double IgapQ = 0.0;
    for (int64_t p = 0; p < S->n;) {
        int s = S->sp[p];
        if (s != SP_E && !heavy_step) { ++p; continue; }
        double dts = (s == SP_E) ? dte : dth;
        real qmdt = R_((double)ZQ[s] * QE / species_mass(s) * dts);
        real dtz = R_(dts / S->c.dz), dtr = R_(dts / S->c.dr);
        int out = push_one(S, p, qmdt, dtz, dtr);
        if (out) {
            int el = out - 1;
            if (S->c.sputter && el < 2 && ZQ[s] > 0) sputter_record(S, p, el);
            S->absorbed[el][s] += 1;
            S->absorbed_energy[el] += S->c.weight * kinetic(S, p);
            /* gap current leaves the anode node: an arriving charge z e W lowers it */
            if (el == 1) IgapQ += -(double)ZQ[s] * QE * S->c.weight;
            /* charge carried through the cathode: emitted electrons add e W (in
             * inject), a returning electron takes it back, an arriving ion adds z e W */
            if (el == 0) S->charge_cathode += (double)ZQ[s] * QE * S->c.weight;
            remove_particle(S, p);
            continue;
        }
        ++p;
    }
    S->I_gap = IgapQ / dte;
}

static void deposit_all(or_sim* S, int heavy_step) {
    int64_t nn = (int64_t)S->nzn * S->nrn;
    memset(S->rho_e, 0, nn * 8);
    if (heavy_step) memset(S->rho_h, 0, nn * 8);
#ifdef OR_OMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t p = 0; p < S->n; ++p) {
        int s = S->sp[p];
        if (s == SP_E) deposit_one(S, S->rho_e, S->iz[p], S->ir[p], S->pz[p], S->pr[p], -1);
        else if (heavy_step && ZQ[s] != 0) deposit_one(S, S->rho_h, S->iz[p], S->ir[p], S->pz[p], S->pr[p], ZQ[s]);
    }
}

/* ------------------------------------------------------------------ */
/* collision kinematics, Eq. (5)-(7) and Eq. (12)-(20)                     */
/* ------------------------------------------------------------------ */
typedef struct { real x, y, z; } vec3;

/* isotropic unit vector, Marsaglia (1972): (a, b) uniform in the unit disc,
 * n = (2a sqrt(1-s), 2b sqrt(1-s), 1-2s) with s = a^2 + b^2. */
static vec3 iso_dir(or_sim* S, stream_t* st) {
    for (int a = 0; a < 64; ++a) {
        real u1 = R_(2) * u01(st) - R_(1);
        real u2 = R_(2) * u01(st) - R_(1);
        real s = u1 * u1 + u2 * u2;
        if (s < R_(1)) {
            real q = R_(2) * OR_SQRT(R_(1) - s);
            vec3 n = {u1 * q, u2 * q, R_(1) - R_(2) * s};
            return n;
        }
    }
    OR_ATOMIC S->iso_fallback++;
    vec3 n = {0, 0, 1};
    return n;
}

/* uniform azimuth psi as (cos psi, sin psi) from a point in the unit disc */
static void azimuth(or_sim* S, stream_t* st, real* c, real* s) {
    for (int a = 0; a < 64; ++a) {
        real u1 = R_(2) * u01(st) - R_(1);
        real u2 = R_(2) * u01(st) - R_(1);
        real q = u1 * u1 + u2 * u2;
        if (q < R_(1) && q > R_(0)) {
            real r = OR_SQRT(q);
            *c = u1 / r; *s = u2 / r;
            return;
        }
    }
    OR_ATOMIC S->iso_fallback++;
    *c = 1; *s = 0;
}

/* Binary collision with energy change: Eq. (6) sets |u'|^2 = |u|^2 + 2 dE/m_r
 * (dE = -E_th, passed as kth = 2 E_th / m_r), the direction of u' is isotropic
 * (Eq. (7) with isotropic I), and Eq. (5) shares u' - u by the reduced mass
 * (a1 = m_r/m1, a2 = m_r/m2).  Returns 0 if the energy is below threshold. */
static int binary_scatter(or_sim* S, stream_t* st, vec3* v1, vec3* v2, real kth, real a1, real a2) {
    vec3 u = {v1->x - v2->x, v1->y - v2->y, v1->z - v2->z};
    real g2 = (u.x * u.x + u.y * u.y) + u.z * u.z;
    real up2 = g2 - kth;
    if (up2 < R_(0)) return 0;
    real gp = OR_SQRT(up2);
    vec3 n = iso_dir(S, st);
    vec3 du = {gp * n.x - u.x, gp * n.y - u.y, gp * n.z - u.z};
    v1->x = v1->x + du.x * a1; v1->y = v1->y + du.y * a1; v1->z = v1->z + du.z * a1;
    v2->x = v2->x - du.x * a2; v2->y = v2->y - du.y * a2; v2->z = v2->z - du.z * a2;
    return 1;
}

/* ------------------------------------------------------------------ */
/* Coulomb collisions (the paper lists them among the collisions of its  */
/* model, Sec. 2.3, without a method): the binary collision model of     */
/* Takizuka and Abe (J. Comput. Phys. 25, 205, 1977).  A pair (a, b)      */
/* with relative velocity u is deflected by theta, tan(theta/2) = delta,  */
/* delta normal with variance <delta^2> = (q_a q_b)^2 n_L lnL dt /        */
/* (8 pi eps0^2 m_ab^2 u^3), about a uniform azimuth; |u| is kept and      */
/* the change of u is shared by the reduced mass, so momentum and energy  */
/* are conserved.  Kn = (q_a q_b)^2 n_L lnL dt / (8 pi eps0^2 m_ab^2) is   */
/* the pair's factor; fa = m_ab / m_a, fb = m_ab / m_b.                   */
/* ------------------------------------------------------------------ */
/* normal deviate approximated by the Irwin-Hall sum of twelve uniforms   */
/* (mean 0, variance 1, support [-6, 6])                                  */
static real irwin_hall12(stream_t* st) {
    real z = R_(0);
    for (int i = 0; i < 12; ++i) z = z + u01(st);
    return z - R_(6);
}

static int coulomb_kin(or_sim* S, stream_t* st, vec3* va, vec3* vb, real Kn, real fa, real fb) {
    real ux = va->x - vb->x, uy = va->y - vb->y, uz = va->z - vb->z;
    real u2 = (ux * ux + uy * uy) + uz * uz;
    if (!(u2 > R_(0))) return 0;
    real u = OR_SQRT(u2);
    real var = Kn / (u2 * u);
    var = var < R_(1e30) ? var : R_(1e30);          /* u -> 0: keep delta finite */
    real z = irwin_hall12(st);
    real d = OR_SQRT(var) * z;
    /* sin(theta) = 2 delta / (1 + delta^2), 1 - cos(theta) = 2 delta^2 / (1 + delta^2),
     * in 1/delta when |delta| > 1 */
    real sth, omc;
    real ad = d < R_(0) ? -d : d;
    if (ad <= R_(1)) {
        real d2 = d * d, den = R_(1) + d2;
        sth = (R_(2) * d) / den;
        omc = (R_(2) * d2) / den;
    } else {
        real r = R_(1) / d, r2 = r * r, den = R_(1) + r2;
        sth = (R_(2) * r) / den;
        omc = R_(2) / den;
    }
    real cph, sph;
    azimuth(S, st, &cph, &sph);
    real sc = sth * cph, ss = sth * sph;
    real up = OR_SQRT(ux * ux + uy * uy);
    real dx, dy, dz;
    if (up > R_(0)) {
        real a1 = ux / up, a2 = uy / up;
        dx = ((a1 * uz) * sc - (a2 * u) * ss) - ux * omc;
        dy = ((a2 * uz) * sc + (a1 * u) * ss) - uy * omc;
        dz = -(up * sc) - uz * omc;
    } else {            /* u along the third axis: rotate about it */
        dx = uz * sc;
        dy = uz * ss;
        dz = -(uz * omc);
    }
    va->x = va->x + fa * dx; va->y = va->y + fa * dy; va->z = va->z + fa * dz;
    vb->x = vb->x - fb * dx; vb->y = vb->y - fb * dy; vb->z = vb->z - fb * dz;
    return 1;
}

static int coulomb_pair(or_sim* S, stream_t* st, int64_t ia, int64_t ib, real Kn, real fa, real fb) {
    vec3 va = {S->vz[ia], S->vr[ia], S->vt[ia]}, vb = {S->vz[ib], S->vr[ib], S->vt[ib]};
    if (!coulomb_kin(S, st, &va, &vb, Kn, fa, fb)) return 0;
    S->vz[ia] = va.x; S->vr[ia] = va.y; S->vt[ia] = va.z;
    S->vz[ib] = vb.x; S->vr[ib] = vb.y; S->vt[ib] = vb.z;
    return 1;
}

/* Pseudo-random permutation of [0, n): a four-round Feistel network
 * (Luby and Rackoff) on 2h bits, 4^h >= n, with an integer mixing round
 * function, walked back into [0, n) by cycle walking (Black and Rogaway,
 * 2002); the walk ends within 4^h steps because x itself lies in [0, n). */
static uint32_t fe_round(uint32_t x, uint32_t k) {
    uint32_t t = (x ^ k) * 0x9E3779B1u;
    t ^= t >> 15;
    t *= 0x85EBCA77u;
    t ^= t >> 13;
    return t;
}
static uint32_t perm_index(uint32_t x, uint32_t n, const uint32_t* key) {
    int h = 1;
    while ((1ull << (2 * h)) < (uint64_t)n) ++h;
    uint32_t mask = (1u << h) - 1u;
    uint64_t lim = 1ull << (2 * h);
    uint32_t y = x;
    for (uint64_t it = 0; it < lim; ++it) {
        uint32_t L = y >> h, R = y & mask;
        for (int r = 0; r < 4; ++r) {
            uint32_t F = fe_round(R, key[r]) & mask;
            uint32_t t = L ^ F;
            L = R;
            R = t;
        }
        y = (L << h) | R;
        if (y < n) return y;
    }
    return x;
}

/* Stage 4 of the double-ionization scheme, Eq. (15)-(20): the velocity v of
 * e3 is the diagonal of a rectangle whose edges are v5 and v6.  v5 =
 * R^-1(theta,phi) R^-1(chi,psi) R(theta,phi) (cos chi v), with R of Eq. (20),
 * which equals cos chi |v| R^T(theta,phi) (sin chi cos psi, sin chi sin psi,
 * cos chi); v6 = v - v5.  theta, phi from the components of v (no angles). */
static void rectangle_split(or_sim* S, stream_t* st, vec3 v, vec3* v5, vec3* v6) {
    real cchi = u01(st);
    if (S->c.di_split_mode == 1) cchi = OR_SQRT(cchi);
    real schi = OR_SQRT(R_(1) - cchi * cchi);
    real cpsi, spsi;
    azimuth(S, st, &cpsi, &spsi);
    real vperp2 = v.x * v.x + v.y * v.y;
    real vmag2 = vperp2 + v.z * v.z;
    real vmag = OR_SQRT(vmag2), vperp = OR_SQRT(vperp2);
    vec3 w5 = {0, 0, 0};
    if (vmag > R_(0)) {
        real ct = v.z / vmag, st_ = vperp / vmag;
        real cp = R_(1), sp = R_(0);
        if (vperp > R_(0)) { cp = v.x / vperp; sp = v.y / vperp; }
        real a = cchi * vmag;                 /* Eq. (16): |alpha v| */
        real w1 = a * (schi * cpsi), w2 = a * (schi * spsi), w3 = a * cchi;  /* Eq. (18) */
        /* Eq. (19): R^T(theta, phi) w, rows of Eq. (20) as columns */
        w5.x = (w1 * (ct * cp) - w2 * sp) + w3 * (st_ * cp);
        w5.y = (w1 * (ct * sp) + w2 * cp) + w3 * (st_ * sp);
        w5.z = w3 * ct - w1 * st_;
    }
    *v5 = w5;
    v6->x = v.x - w5.x; v6->y = v.y - w5.y; v6->z = v.z - w5.z;
}

/* One accepted event of channel ch between electron ie and heavy it (ids of
 * spawned electrons come from *next_id).  Returns the number of spawned
 * electrons, or -1 if the energy was below threshold (no event). */
static int collide_event(or_sim* S, stream_t* st, int ch, int64_t ie, int64_t it,
                         uint32_t* next_id, int64_t* rho_e, int64_t* rho_h) {
    double mr = mr_class();
    real a_e = R_(mr / ME), a_t = R_(mr / M_CU);
    real kth = R_(2.0 * S->eth[ch] * QE / mr);
    vec3 ve = {S->vz[ie], S->vr[ie], S->vt[ie]};
    vec3 vt = {S->vz[it], S->vr[it], S->vt[it]};
    if (ch == CH_EL || ch == CH_EXC) {
        if (!binary_scatter(S, st, &ve, &vt, ch == CH_EL ? R_(0) : kth, a_e, a_t)) return -1;
        S->vz[ie] = ve.x; S->vr[ie] = ve.y; S->vt[ie] = ve.z;
        S->vz[it] = vt.x; S->vr[it] = vt.y; S->vt[it] = vt.z;
        return 0;
    }
    /* Stage 1, Eq. (12): e + A -> e1 + A*, losing the ionization threshold */
    if (!binary_scatter(S, st, &ve, &vt, kth, a_e, a_t)) return -1;
    /* Stage 2, Eq. (13): A* -> e2 + ion; both inherit position and velocity of A* */
    vec3 e2 = vt;
    /* Stage 3, Eq. (14): e1 + e2 elastic, equal masses (m_r/m = 1/2) */
    binary_scatter(S, st, &ve, &e2, R_(0), R_(0.5), R_(0.5));
    int new_sp = ch == CH_SI ? SP_CUP
               : ch == CH_SW ? SP_CU2_SW
               : ch == CH_DI ? SP_CU2_DI
               : ch == CH_S3 ? SP_CU3 : SP_CU4;
    int dz = ZQ[new_sp] - ZQ[S->sp[it]];
    int nspawn = 0;
    vec3 e_keep = ve;
    vec3 e6 = {0, 0, 0};
    if (ch == CH_DI) {
        /* Stage 4, Eq. (15): e3 -> e5 + e6 (velocity rectangle) */
        vec3 e5;
        rectangle_split(S, st, ve, &e5, &e6);
        e_keep = e5;
    }
    /* apply: projectile keeps e3 (SI/SW) or e5 (DI), target becomes the ion */
    S->vz[ie] = e_keep.x; S->vr[ie] = e_keep.y; S->vt[ie] = e_keep.z;
    S->vz[it] = vt.x; S->vr[it] = vt.y; S->vt[it] = vt.z;
    S->sp[it] = (uint8_t)new_sp;
    deposit_one(S, rho_h, S->iz[it], S->ir[it], S->pz[it], S->pr[it], dz);
    /* e2 (scattered into e4) at the position of A* */
    int64_t q = spawn_particle(S, SP_E, S->iz[it], S->ir[it], S->pz[it], S->pr[it], e2.x, e2.y, e2.z, (*next_id)++);
    if (q < 0) return -2;
    deposit_one(S, rho_e, S->iz[it], S->ir[it], S->pz[it], S->pr[it], -1);
    ++nspawn;
    if (ch == CH_DI) {
        /* e6 at the position of e3 (the projectile) */
        q = spawn_particle(S, SP_E, S->iz[ie], S->ir[ie], S->pz[ie], S->pr[ie], e6.x, e6.y, e6.z, (*next_id)++);
        if (q < 0) return -2;
        deposit_one(S, rho_e, S->iz[ie], S->ir[ie], S->pz[ie], S->pr[ie], -1);
        ++nspawn;
    }
    return nspawn;
}

/* exported for the per-event conservation checks: one event of channel ch
 * between velocities ve and vt, drawing from stream (subject, step, sid). */
int or_event_kinematics(or_sim* S, int ch, uint32_t subject, uint32_t step, uint32_t sid,
                        double* ve_io, double* vt_io, double* e_new /* 6 */, int* nspawn) {
    stream_t st;
    stream_init(&st, S, subject, step, sid);
    double mr = mr_class();
    real a_e = R_(mr / ME), a_t = R_(mr / M_CU);
    real kth = R_(2.0 * S->eth[ch] * QE / mr);
    vec3 ve = {R_(ve_io[0]), R_(ve_io[1]), R_(ve_io[2])};
    vec3 vt = {R_(vt_io[0]), R_(vt_io[1]), R_(vt_io[2])};
    *nspawn = 0;
    if (ch == CH_EL || ch == CH_EXC) {
        if (!binary_scatter(S, &st, &ve, &vt, ch == CH_EL ? R_(0) : kth, a_e, a_t)) return -1;
    } else {
        if (!binary_scatter(S, &st, &ve, &vt, kth, a_e, a_t)) return -1;
        vec3 e2 = vt;
        binary_scatter(S, &st, &ve, &e2, R_(0), R_(0.5), R_(0.5));
        e_new[0] = e2.x; e_new[1] = e2.y; e_new[2] = e2.z;
        *nspawn = 1;
        if (ch == CH_DI) {
            vec3 e5, e6;
            rectangle_split(S, &st, ve, &e5, &e6);
            ve = e5;
            e_new[3] = e6.x; e_new[4] = e6.y; e_new[5] = e6.z;
            *nspawn = 2;
        }
    }
    ve_io[0] = ve.x; ve_io[1] = ve.y; ve_io[2] = ve.z;
    vt_io[0] = vt.x; vt_io[1] = vt.y; vt_io[2] = vt.z;
    return 0;
}

/* exported for the pins of the Coulomb model: one pair collision of
 * velocities va, vb with factor Kn and mass fractions fa, fb, drawing from
 * stream (subject, step, sid); the permutation of [0, n) under key[4] */
int or_coulomb_kinematics(or_sim* S, uint32_t subject, uint32_t step, uint32_t sid, double* va_io, double* vb_io,
                          double Kn, double fa, double fb) {
    stream_t st;
    stream_init(&st, S, subject, step, sid);
    vec3 va = {R_(va_io[0]), R_(va_io[1]), R_(va_io[2])}, vb = {R_(vb_io[0]), R_(vb_io[1]), R_(vb_io[2])};
    int r = coulomb_kin(S, &st, &va, &vb, R_(Kn), R_(fa), R_(fb));
    va_io[0] = va.x; va_io[1] = va.y; va_io[2] = va.z;
    vb_io[0] = vb.x; vb_io[1] = vb.y; vb_io[2] = vb.z;
    return r;
}
uint32_t or_perm_index(uint32_t x, uint32_t n, const uint32_t* key) { return perm_index(x, n, key); }

int or_rectangle_split(or_sim* S, uint32_t subject, uint32_t step, uint32_t sid, const double* v,
                       double* v5, double* v6) {
    stream_t st;
    stream_init(&st, S, subject, step, sid);
    vec3 vv = {R_(v[0]), R_(v[1]), R_(v[2])}, a, b;
    rectangle_split(S, &st, vv, &a, &b);
    v5[0] = a.x; v5[1] = a.y; v5[2] = a.z;
    v6[0] = b.x; v6[1] = b.y; v6[2] = b.z;
    return 0;
}

/* ------------------------------------------------------------------ */
/* DSMC collision step, Sec. 2.1 Eq. (4) in no-time-counter form:        */
/* per cell and pair class (e,Cu), (e,Cu+): N_cand = floor(N_e N_t W       */
/* (sigma g)_max dt_coll / V_c + R); each candidate is a random electron   */
/* and a random target of the cell, accepted when R (sigma g)_max <        */
/* sigma_T g, i.e. with the linearised probability of Eq. (4) relative to  */
/* the majorant; the channel is drawn in proportion to sigma_c.            */
/* ------------------------------------------------------------------ */
typedef struct { uint32_t id; int64_t idx; } idrec;
static int cmp_id(const void* a, const void* b) {
    uint32_t x = ((const idrec*)a)->id, y = ((const idrec*)b)->id;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* one species paired with itself: two by two in a random order, an odd
 * count ending with a triple of three pairs at half the time step; a
 * particle whose species changed this step is left out */
static uint64_t pairs_same(or_sim* S, int64_t c, const idrec* l, uint32_t N, int sp, int cls, real Kn, real f) {
    uint64_t done = 0;
    if (N < 2) return 0;
    stream_t ps;
    stream_init(&ps, S, (uint32_t)c, S->step, SID_COUL_PERM(cls));
    uint32_t key[4];
    for (int q = 0; q < 4; ++q) key[q] = next_u32(&ps);
    uint32_t P = N / 2 - (N % 2);                              /* regular pairs */
    for (uint32_t k = 0; k < P; ++k) {
        int64_t ia = l[perm_index(2 * k, N, key)].idx, ib = l[perm_index(2 * k + 1, N, key)].idx;
        if (S->sp[ia] != sp || S->sp[ib] != sp) continue;
        stream_t st;
        stream_init(&st, S, (uint32_t)c, S->step, SID_COUL(cls, k));
        done += (uint64_t)coulomb_pair(S, &st, ia, ib, Kn, f, f);
    }
    if (N % 2) {                                               /* the last three: a triple */
        int64_t t[3];
        for (int q = 0; q < 3; ++q) t[q] = l[perm_index(N - 3 + q, N, key)].idx;
        for (int q = 0; q < 3; ++q) {
            int64_t ia = t[q], ib = t[(q + 1) % 3];
            if (S->sp[ia] != sp || S->sp[ib] != sp) continue;
            stream_t st;
            stream_init(&st, S, (uint32_t)c, S->step, SID_COUL(cls, P + (uint32_t)q));
            done += (uint64_t)coulomb_pair(S, &st, ia, ib, Kn * R_(0.5), f, f);
        }
    }
    return done;
}

/* two species A and B: each particle of the more numerous (A on a tie) once,
 * the k-th of it in a random order with the (k mod N_fewer)-th of the other
 * in a random order, so that a particle of the fewer collides several times
 * in sequence; the first particle of every pair is A's */
static uint64_t pairs_cross(or_sim* S, int64_t c, const idrec* la, uint32_t NA, int spa, const idrec* lb,
                            uint32_t NB, int spb, int cls, real Kn, real fa, real fb) {
    uint64_t done = 0;
    if (NA == 0 || NB == 0) return 0;
    int a_many = NA >= NB;
    uint32_t Nm = a_many ? NA : NB, Nf = a_many ? NB : NA;
    stream_t ps;
    stream_init(&ps, S, (uint32_t)c, S->step, SID_COUL_PERM(cls));
    uint32_t km[4], kf[4];
    for (int q = 0; q < 4; ++q) km[q] = next_u32(&ps);
    for (int q = 0; q < 4; ++q) kf[q] = next_u32(&ps);
    for (uint32_t k = 0; k < Nm; ++k) {
        uint32_t m = perm_index(k, Nm, km), f = perm_index(k % Nf, Nf, kf);
        int64_t ia = a_many ? la[m].idx : la[f].idx;
        int64_t ib = a_many ? lb[f].idx : lb[m].idx;
        if (S->sp[ia] != spa || S->sp[ib] != spb) continue;   /* ionized this step */
        stream_t st;
        stream_init(&st, S, (uint32_t)c, S->step, SID_COUL(cls, k));
        done += (uint64_t)coulomb_pair(S, &st, ia, ib, Kn, fa, fb);
    }
    return done;
}

/* Pairing of one cell (Takizuka-Abe), on the lists of the step's start:
 * class 0 pairs the electrons with themselves, class 1 + i the electrons
 * with ion species i (Cu+, Cu2+ SW, Cu2+ DI, Cu3+, Cu4+), both with the
 * electron collision step; on heavy steps, classes 6.. pair the ion species
 * with themselves and with each other (species a <= b in order), with the
 * heavy step.  n_L is the density of the fewer of the two (of the species
 * itself in a class of one species). */
static double coulomb_k(int za, int zb, double mab, double lnl) {
    double qq = (double)za * (double)zb * QE * QE;
    return qq * qq * lnl / (8.0 * PI * EPS0 * EPS0 * mab * mab);
}

static void coulomb_cell(or_sim* S, int64_t c, const idrec* rec, const int64_t* cnt, int64_t C, double dtc,
                         int heavy_step) {
    int j = (int)(c % S->c.nr);
    double wv = S->c.weight * dtc / cell_volume(S, j);          /* W dt / V: n dt per particle */
    double lnl = S->c.coulomb_lnl;
    const idrec* el = rec + cnt[SP_E * C + c];
    uint32_t Ne = (uint32_t)(cnt[SP_E * C + c + 1] - cnt[SP_E * C + c]);
    uint64_t ee_ = pairs_same(S, c, el, Ne, SP_E, 0, R_(coulomb_k(-1, -1, 0.5 * ME, lnl) * (double)Ne * wv), R_(0.5));
    OR_ATOMIC S->coul_ee += ee_;
    double mr = mr_class();
    real fe = R_(mr / ME), fi = R_(mr / M_CU);
    const idrec* il[5];
    uint32_t Ni[5];
    for (int i = 0; i < 5; ++i) {
        int sp = SP_CUP + i;
        il[i] = rec + cnt[sp * C + c];
        Ni[i] = (uint32_t)(cnt[sp * C + c + 1] - cnt[sp * C + c]);
    }
    for (int i = 0; i < 5; ++i) {
        uint32_t Nf = Ne < Ni[i] ? Ne : Ni[i];
        real Kn = R_(coulomb_k(-1, ZQ[SP_CUP + i], mr, lnl) * (double)Nf * wv);
        uint64_t ei_ = pairs_cross(S, c, el, Ne, SP_E, il[i], Ni[i], SP_CUP + i, 1 + i, Kn, fe, fi);
        OR_ATOMIC S->coul_ei += ei_;
    }
    if (!heavy_step) return;
    double wvh = S->c.weight * (dtc * S->c.heavy_subcycle) / cell_volume(S, j);
    int cls = 6;
    for (int a = 0; a < 5; ++a)
        for (int b = a; b < 5; ++b, ++cls) {
            int sa = SP_CUP + a, sb = SP_CUP + b;
            uint32_t Nf = a == b ? Ni[a] : (Ni[a] < Ni[b] ? Ni[a] : Ni[b]);
            real Kn = R_(coulomb_k(ZQ[sa], ZQ[sb], 0.5 * M_CU, lnl) * (double)Nf * wvh);
            uint64_t ii_ = a == b ? pairs_same(S, c, il[a], Ni[a], sa, cls, Kn, R_(0.5))
                                  : pairs_cross(S, c, il[a], Ni[a], sa, il[b], Ni[b], sb, cls, Kn, R_(0.5), R_(0.5));
            OR_ATOMIC S->coul_ii += ii_;
        }
}

static int collide_all(or_sim* S, int heavy_step) {
    int64_t C = (int64_t)S->c.nz * S->c.nr;
    int64_t nb = C * NSP;
    int64_t* cnt = (int64_t*)calloc(nb + 1, 8);
    int64_t n0 = S->n;
#ifdef OR_OMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t p = 0; p < n0; ++p) {
        int64_t cell = (int64_t)S->iz[p] * S->c.nr + S->ir[p];
        OR_ATOMIC cnt[(int64_t)S->sp[p] * C + cell + 1]++;
    }
    for (int64_t b = 0; b < nb; ++b) cnt[b + 1] += cnt[b];
    idrec* rec = (idrec*)malloc((n0 > 0 ? n0 : 1) * sizeof(idrec));
    int64_t* cur = (int64_t*)malloc((nb > 0 ? nb : 1) * 8);
    memcpy(cur, cnt, nb * 8);
#ifdef OR_OMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t p = 0; p < n0; ++p) {
        int64_t cell = (int64_t)S->iz[p] * S->c.nr + S->ir[p];
        int64_t b = (int64_t)S->sp[p] * C + cell;
        int64_t at;
#ifdef OR_OMP
#pragma omp atomic capture
#endif
        at = cur[b]++;
        rec[at].id = S->id[p];
        rec[at].idx = p;
    }
    /* canonical order inside each (species, cell) bin: ascending id */
#ifdef OR_OMP
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (int64_t b = 0; b < nb; ++b)
        if (cnt[b + 1] - cnt[b] > 1) qsort(rec + cnt[b], cnt[b + 1] - cnt[b], sizeof(idrec), cmp_id);

    /* candidate counts per cell and their prefix sum (spawn id slots: the
     * electron classes only; heavy pairs spawn nothing).  The cell's stream
     * gives R_k to class k, k = 0..6, whether the class is on or not. */
    uint32_t* nc = (uint32_t*)calloc(NCLS * C, 4);
    uint64_t total = 0, heavy_total = 0;
    uint64_t* pre = (uint64_t*)malloc((C + 1) * 8);
    double dtc = S->c.dt * S->c.coll_dt_scale;
    double dth = dtc * S->c.heavy_subcycle;                 /* heavy pairs collide on heavy steps */
    int heavy = S->c.heavy_coll && heavy_step;
#ifdef OR_OMP
#pragma omp parallel for schedule(static) reduction(+ : total, heavy_total)
#endif
    for (int64_t c = 0; c < C; ++c) {
        int j = (int)(c % S->c.nr);
        stream_t st;
        stream_init(&st, S, (uint32_t)c, S->step, SID_NCAND);
        uint32_t Ne = (uint32_t)(cnt[SP_E * C + c + 1] - cnt[SP_E * C + c]);
        uint32_t Ncu = (uint32_t)(cnt[SP_CU * C + c + 1] - cnt[SP_CU * C + c]);
        uint32_t Ni = (uint32_t)(cnt[SP_CUP * C + c + 1] - cnt[SP_CUP * C + c]);
        real R[NCLS];
        for (int k = 0; k < NCLS; ++k) R[k] = u01(&st);
        for (int k = 0; k < NECLS; ++k) {
            if (CLASS_QMAX[k] > S->c.charge_max) continue;
            int ts = CLASS_TARGET[k];
            uint32_t Nt = (uint32_t)(cnt[ts * C + c + 1] - cnt[ts * C + c]);
            real ck = R_(S->c.weight * (double)S->sgmax[k] * dtc / cell_volume(S, j));
            real x = ((real)Ne * (real)Nt) * ck + R[k];
            nc[NCLS * c + k] = (uint32_t)OR_FLOOR(x);
            total += nc[NCLS * c + k];
        }
        if (heavy) {
            /* N_cu N_cu+ pairs for charge exchange, N_cu (N_cu - 1) / 2 for Cu-Cu */
            real ck5 = R_(S->c.weight * (double)S->sgmax[5] * dth / cell_volume(S, j));
            real ck6 = R_(0.5 * S->c.weight * (double)S->sgmax[6] * dth / cell_volume(S, j));
            real x5 = ((real)Ncu * (real)Ni) * ck5 + R[5];
            real x6 = ((real)Ncu * (real)(Ncu > 0 ? Ncu - 1 : 0)) * ck6 + R[6];
            nc[NCLS * c + 5] = (uint32_t)OR_FLOOR(x5);
            nc[NCLS * c + 6] = (uint32_t)OR_FLOOR(x6);
            if (Ncu < 2) nc[NCLS * c + 6] = 0;
            heavy_total += nc[NCLS * c + 5] + nc[NCLS * c + 6];
        }
    }
    /* spawn id slots of each cell: prefix of its electron-class candidates */
    {
        uint64_t acc = 0;
        for (int64_t c = 0; c < C; ++c) {
            pre[c] = acc;
            for (int k = 0; k < NECLS; ++k) acc += nc[NCLS * c + k];
        }
    }
    pre[C] = total;
    S->cand_total += total + heavy_total;
    uint32_t id_base = S->id_next;
    real km = kmr(), kmh = kmr_heavy();
    int err = 0;
#ifdef OR_OMP
    /* cells in parallel, each cell's spawns in the slots of its ids; only
     * when the reserved slots fit (the serial order otherwise) */
    const int par = S->n + 2 * (int64_t)total <= S->cap;
    if (par) {
        S->spawn_mode = 1;
        S->spawn_base = S->n;
        S->spawn_id0 = id_base;
        for (int64_t q = S->n; q < S->n + 2 * (int64_t)total; ++q) S->sp[q] = 255;
    }
#pragma omp parallel for schedule(dynamic, 64) if (par)
#endif
    for (int64_t c = 0; c < C; ++c) {
        if (err) continue;
        uint32_t next_id = id_base + (uint32_t)(2 * pre[c]);
        const idrec* el = rec + cnt[SP_E * C + c];
        uint32_t Ne = (uint32_t)(cnt[SP_E * C + c + 1] - cnt[SP_E * C + c]);
        const idrec* cul = rec + cnt[SP_CU * C + c];
        uint32_t Ncu = (uint32_t)(cnt[SP_CU * C + c + 1] - cnt[SP_CU * C + c]);
        for (int k = 0; k < NECLS && !err; ++k) {
            int ts = CLASS_TARGET[k];
            const idrec* tl = rec + cnt[ts * C + c];
            uint32_t Nt = (uint32_t)(cnt[ts * C + c + 1] - cnt[ts * C + c]);
            for (uint32_t m = 0; m < nc[NCLS * c + k]; ++m) {
                stream_t st;
                stream_init(&st, S, (uint32_t)c, S->step, SID_CAND(k, m));
                uint32_t i = pick(&st, Ne), jt = pick(&st, Nt);
                real Racc = u01(&st), Rch = u01(&st);
                int64_t ie = el[i].idx, it = tl[jt].idx;
                if (S->sp[it] != ts) { OR_ATOMIC S->consumed++; continue; }   /* target already ionized this step */
                real ux = S->vz[ie] - S->vz[it], uy = S->vr[ie] - S->vr[it], uz = S->vt[ie] - S->vt[it];
                real g2 = (ux * ux + uy * uy) + uz * uz;
                real g = OR_SQRT(g2);
                real eps = g2 * km;
                real cum[4];
                real sT = 0;
                for (int q = 0; q < CLASS_NCH[k]; ++q) {
                    sT = sT + xs_lookup(S, CLASS_CH0[k] + q, eps);
                    cum[q] = sT;
                }
                real sg = sT * g;
                if (sg > S->sgmax[k]) { OR_ATOMIC S->ratio_viol++; }
                if (!(Racc * S->sgmax[k] < sg)) { OR_ATOMIC S->nulls++; continue; }
                real rs = Rch * sT;
                int q = -1;
                for (int a = 0; a < CLASS_NCH[k]; ++a) if (rs < cum[a]) { q = a; break; }
                if (q < 0) {   /* defensive: last channel with a positive share */
                    q = CLASS_NCH[k] - 1;
                    for (int a = CLASS_NCH[k] - 1; a >= 0; --a)
                        if (cum[a] > (a ? cum[a - 1] : R_(0))) { q = a; break; }
                }
                int ch = CLASS_CH0[k] + q;
                int r = collide_event(S, &st, ch, ie, it, &next_id, S->rho_e, S->rho_h);
                if (r == -2) { err = 1; break; }
                if (r < 0) { OR_ATOMIC S->thr_rej++; continue; }
                OR_ATOMIC S->events[ch]++;
            }
        }
        /* heavy pairs, classes 5 (Cu from the Cu list, Cu+ from the Cu+ list) and
         * 6 (two different Cu of the Cu list); a particle whose species changed
         * this step (ionized) is consumed */
        for (int k = NECLS; k < NCLS && heavy && !err; ++k) {
            int ts = CLASS_TARGET[k];
            const idrec* tl = rec + cnt[ts * C + c];
            uint32_t Nt = (uint32_t)(cnt[ts * C + c + 1] - cnt[ts * C + c]);
            for (uint32_t m = 0; m < nc[NCLS * c + k]; ++m) {
                stream_t st;
                stream_init(&st, S, (uint32_t)c, S->step, SID_CAND(k, m));
                uint32_t i = pick(&st, Ncu), jt;
                if (k == 5) jt = pick(&st, Nt);
                else {          /* a second, different Cu */
                    jt = pick(&st, Ncu - 1);
                    if (jt >= i) jt++;
                }
                real Racc = u01(&st);
                (void)u01(&st);     /* fourth draw of the candidate, unused by one-channel classes */
                int64_t ia = cul[i].idx, ib = tl[jt].idx;
                if (S->sp[ia] != SP_CU || S->sp[ib] != ts) { OR_ATOMIC S->consumed++; continue; }
                real ux = S->vz[ia] - S->vz[ib], uy = S->vr[ia] - S->vr[ib], uz = S->vt[ia] - S->vt[ib];
                real g2 = (ux * ux + uy * uy) + uz * uz;
                real g = OR_SQRT(g2);
                real sg = xs_lookup(S, CLASS_CH0[k], g2 * kmh) * g;
                if (sg > S->sgmax[k]) { OR_ATOMIC S->ratio_viol++; }
                if (!(Racc * S->sgmax[k] < sg)) { OR_ATOMIC S->nulls++; continue; }
                if (k == 5) {
                    /* resonant charge exchange: the electron moves to the ion, the
                     * velocities stay with the atoms: the Cu+ slot takes the Cu's
                     * velocity and the Cu slot the ion's */
                    real t;
                    t = S->vz[ia]; S->vz[ia] = S->vz[ib]; S->vz[ib] = t;
                    t = S->vr[ia]; S->vr[ia] = S->vr[ib]; S->vr[ib] = t;
                    t = S->vt[ia]; S->vt[ia] = S->vt[ib]; S->vt[ib] = t;
                } else {
                    /* elastic, equal masses (m_r/m = 1/2), isotropic in the centre of mass */
                    vec3 va = {S->vz[ia], S->vr[ia], S->vt[ia]};
                    vec3 vb = {S->vz[ib], S->vr[ib], S->vt[ib]};
                    binary_scatter(S, &st, &va, &vb, R_(0), R_(0.5), R_(0.5));
                    S->vz[ia] = va.x; S->vr[ia] = va.y; S->vt[ia] = va.z;
                    S->vz[ib] = vb.x; S->vr[ib] = vb.y; S->vt[ib] = vb.z;
                }
                OR_ATOMIC S->events[CLASS_CH0[k]]++;
            }
        }
        /* Coulomb collisions of the cell's charged particles, after its DSMC
         * classes: e-e, then e with each ion species.  The lists are those of
         * the step's start (newborn electrons wait for the next step); an ion
         * ionized earlier this step is left out. */
        if (S->c.coulomb && !err) coulomb_cell(S, c, rec, cnt, C, dtc, heavy_step);
    }
#ifdef OR_OMP
    if (par) {
        /* the reserved slots, compacted in order: the serial build's appends */
        int64_t w = S->n, end = S->n + 2 * (int64_t)total;
        for (int64_t q = S->n; q < end; ++q) {
            if (S->sp[q] == 255) continue;
            if (q != w) {
                S->sp[w] = S->sp[q]; S->iz[w] = S->iz[q]; S->ir[w] = S->ir[q];
                S->pz[w] = S->pz[q]; S->pr[w] = S->pr[q];
                S->vz[w] = S->vz[q]; S->vr[w] = S->vr[q]; S->vt[w] = S->vt[q];
                S->id[w] = S->id[q];
            }
            ++w;
        }
        S->n = w;
        S->spawn_mode = 0;
    }
#endif
    S->id_next = id_base + (uint32_t)(2 * total);
    free(cnt); free(rec); free(cur); free(nc); free(pre);
    return err;
}

/* ------------------------------------------------------------------ */
/* Poisson, Eq. (8) read as lap(phi) = -rho/eps0, finite volumes on the   */
/* r-z node grid: Dirichlet phi = 0 at the cathode (z = 0) and V at the   */
/* anode (z = L), symmetry on the axis, Neumann at r = R.  The node       */
/* charge density rho_j = Q_j / V_j (Verboncoeur volumes) enters as       */
/* rho_j times the finite-volume control volume.  Solved by conjugate      */
/* gradients in double to a relative residual below tol.                   */
/* ------------------------------------------------------------------ */
typedef struct { double ap, am, b, vfv; } rzcoef;

static void rz_coefs(const or_sim* S, rzcoef* cf) {
    int N = S->c.nr;
    double dz = S->c.dz, dr = S->c.dr, R = N * dr;
    for (int j = 0; j <= N; ++j) {
        double rp = (j + 0.5) * dr, rm = (j - 0.5) * dr;
        cf[j].ap = (j < N) ? 2.0 * PI * rp * dz / dr : 0.0;
        cf[j].am = (j > 0) ? 2.0 * PI * rm * dz / dr : 0.0;
        double A;
        if (j == 0) A = PI * (0.5 * dr) * (0.5 * dr);
        else if (j == N) A = PI * (R * R - (R - 0.5 * dr) * (R - 0.5 * dr));
        else A = 2.0 * PI * j * dr * dr;
        cf[j].b = A / dz;
        cf[j].vfv = A * dz;
    }
}

static void rz_apply(const or_sim* S, const rzcoef* cf, const double* x, double* y) {
    int NZ = S->c.nz, NR = S->c.nr, W = NR + 1;
    for (int i = 1; i < NZ; ++i)
        for (int j = 0; j <= NR; ++j) {
            double xc = x[i * W + j];
            double s = (cf[j].ap + cf[j].am + 2.0 * cf[j].b) * xc;
            if (j < NR) s -= cf[j].ap * x[i * W + j + 1];
            if (j > 0) s -= cf[j].am * x[i * W + j - 1];
            if (i + 1 < NZ) s -= cf[j].b * x[(i + 1) * W + j];
            if (i - 1 > 0) s -= cf[j].b * x[(i - 1) * W + j];
            y[i * W + j] = s;
        }
}

/* rho: node charge density (C/m^3); Vanode: anode potential.  phi is the
 * initial guess on entry and the solution on exit (electrode rows set). */
int or_poisson_solve(or_sim* S, const double* rho, double Vanode, double tol, double* phi) {
    int NZ = S->c.nz, NR = S->c.nr, W = NR + 1;
    int64_t nn = (int64_t)(NZ + 1) * W;
    rzcoef* cf = (rzcoef*)malloc(W * sizeof(rzcoef));
    rz_coefs(S, cf);
    double *b = calloc(nn, 8), *r = calloc(nn, 8), *p = calloc(nn, 8), *Ap = calloc(nn, 8), *x = calloc(nn, 8);
    for (int i = 1; i < NZ; ++i)
        for (int j = 0; j <= NR; ++j) {
            double v = rho[i * W + j] * cf[j].vfv / EPS0;
            if (i == NZ - 1) v += cf[j].b * Vanode;
            b[i * W + j] = v;
            x[i * W + j] = phi[i * W + j];
        }
    double bn = 0;
    for (int64_t k = 0; k < nn; ++k) bn += b[k] * b[k];
    bn = sqrt(bn);
    rz_apply(S, cf, x, Ap);
    double rr = 0;
    for (int i = 1; i < NZ; ++i)
        for (int j = 0; j <= NR; ++j) {
            int64_t k = (int64_t)i * W + j;
            r[k] = b[k] - Ap[k];
            p[k] = r[k];
            rr += r[k] * r[k];
        }
    int it = 0;
    int maxit = 20 * (NZ + NR) * 10 + 1000;
    while (bn > 0 && sqrt(rr) > tol * bn && it < maxit) {
        rz_apply(S, cf, p, Ap);
        double pAp = 0;
        for (int i = 1; i < NZ; ++i)
            for (int j = 0; j <= NR; ++j) { int64_t k = (int64_t)i * W + j; pAp += p[k] * Ap[k]; }
        double alpha = rr / pAp;
        double rr2 = 0;
        for (int i = 1; i < NZ; ++i)
            for (int j = 0; j <= NR; ++j) {
                int64_t k = (int64_t)i * W + j;
                x[k] += alpha * p[k];
                r[k] -= alpha * Ap[k];
                rr2 += r[k] * r[k];
            }
        double beta = rr2 / rr;
        rr = rr2;
        for (int i = 1; i < NZ; ++i)
            for (int j = 0; j <= NR; ++j) { int64_t k = (int64_t)i * W + j; p[k] = r[k] + beta * p[k]; }
        ++it;
    }
    for (int j = 0; j <= NR; ++j) { x[j] = 0.0; x[NZ * W + j] = Vanode; }
    /* true residual of the final iterate */
    rz_apply(S, cf, x, Ap);
    double tr = 0;
    for (int i = 1; i < NZ; ++i)
        for (int j = 0; j <= NR; ++j) {
            int64_t k = (int64_t)i * W + j;
            double bb = rho[k] * cf[j].vfv / EPS0;
            double ax = Ap[k];
            if (i == NZ - 1) bb += cf[j].b * Vanode;
            tr += (bb - ax) * (bb - ax);
        }
    memcpy(phi, x, nn * 8);
    S->poisson_iters = it;
    S->poisson_relres = bn > 0 ? sqrt(tr) / bn : 0.0;
    free(cf); free(b); free(r); free(p); free(Ap); free(x);
    return it;
}

/* E = -grad(phi) on the nodes: central differences inside, one-sided at the
 * electrodes, E_r = 0 on the axis and at r = R (symmetry / Neumann). */
void or_efield(const or_sim* S, const double* phi, double* Ez, double* Er) {
    int NZ = S->c.nz, NR = S->c.nr, W = NR + 1;
    double dz = S->c.dz, dr = S->c.dr;
    for (int i = 0; i <= NZ; ++i)
        for (int j = 0; j <= NR; ++j) {
            int64_t k = (int64_t)i * W + j;
            if (i == 0) Ez[k] = -(phi[k + W] - phi[k]) / dz;
            else if (i == NZ) Ez[k] = -(phi[k] - phi[k - W]) / dz;
            else Ez[k] = -(phi[k + W] - phi[k - W]) / (2.0 * dz);
            if (j == 0 || j == NR) Er[k] = 0.0;
            else Er[k] = -(phi[k + 1] - phi[k - 1]) / (2.0 * dr);
        }
}

/* node charge density (C/m^3) from fixed-point charge */
static void rho_density(const or_sim* S, double* rho) {
    double f = QE * S->c.weight / 4294967296.0;
    for (int i = 0; i < S->nzn; ++i)
        for (int j = 0; j < S->nrn; ++j) {
            int64_t k = (int64_t)i * S->nrn + j;
            rho[k] = f * (double)(S->rho_e[k] + S->rho_h[k]) / node_volume(S, i, j);
        }
}

static void field_solve(or_sim* S) {
    int64_t nn = (int64_t)S->nzn * S->nrn;
    double* rho = (double*)malloc(nn * 8);
    double* Ez = (double*)malloc(nn * 8);
    double* Er = (double*)malloc(nn * 8);
    rho_density(S, rho);
    or_poisson_solve(S, rho, S->V, S->c.poisson_tol, S->phi);
    or_efield(S, S->phi, Ez, Er);
    for (int64_t k = 0; k < nn; ++k) { S->Ez[k] = R_(Ez[k]); S->Er[k] = R_(Er[k]); }
    free(rho); free(Ez); free(Er);
}

/* ------------------------------------------------------------------ */
/* cathode injection (Sec. 2.3): Fowler-Nordheim electrons from the tip     */
/* (radius r_tip on the axis, field enhanced by beta) and neutrals at a     */
/* fixed fraction of the electron flux.                                     */
/* ------------------------------------------------------------------ */
/* elementary FN current density J = (A/phi) F^2 exp(-B phi^(3/2) / F), A/m^2 */
double or_fn_current(double F, double work) {
    const double A = 1.541434e-6, B = 6.830890e9;
    if (F <= 0.0) return 0.0;
    return A / work * F * F * exp(-B * work * sqrt(work) / F);
}

static real rayleigh(const or_sim* S, real U) {
    real x = U * R_(1023);
    int k = (int)x;
    real t = x - (real)k;
    return (real)S->ray[k] + t * ((real)S->ray[k + 1] - (real)S->ray[k]);
}

static int inject(or_sim* S) {
    if (S->c.geom != 0 || !S->c.inject_on) return 0;
    double dr = S->c.dr, rt = S->c.tip_radius;
    real rtip_cells = R_(rt / dr);
    real vth = R_(sqrt(KB * S->c.neutral_T / M_CU));
    for (int j = 0; (double)j * dr < rt && j < S->c.nr; ++j) {
        double rhi = fmin((j + 1) * dr, rt), rlo = j * dr;
        double area = PI * (rhi * rhi - rlo * rlo);
        double Ezs = 0.5 * ((double)S->Ez[j] + (double)S->Ez[j + 1]);   /* nodes (0,j), (0,j+1) */
        double F = S->c.beta * (Ezs < 0 ? -Ezs : 0.0);
        double J = or_fn_current(F, S->c.work_function);
        double lam_e = J * area * S->c.dt / (QE * S->c.weight);
        double lam_n = S->c.neutral_ratio * lam_e;
        stream_t st;
        stream_init(&st, S, (uint32_t)j, S->step, SID_INJ_COUNT);
        double Re = (double)u01(&st), Rn = (double)u01(&st);
        uint32_t ne = (uint32_t)floor(lam_e + Re), nn = (uint32_t)floor(lam_n + Rn);
        real hi = (j + 1) * dr <= rt ? R_(j + 1) : rtip_cells;
        real lo = R_(j);
        for (uint32_t p = 0; p < ne + nn; ++p) {
            int is_e = p < ne;
            stream_t sp;
            stream_init(&sp, S, (uint32_t)j, S->step, is_e ? SID_INJ_E(p) : SID_INJ_CU(p - ne));
            real U = u01(&sp);
            real rr = OR_SQRT(lo * lo + U * (hi * hi - lo * lo));
            real pr = rr - lo;
            if (pr >= R_(1)) pr = ONE_MINUS_ULP;
            if (pr < R_(0)) pr = R_(0);
            real vz = 0, vr = 0, vt = 0;
            if (!is_e) {
                real U1 = u01(&sp), U2 = u01(&sp);
                vz = vth * rayleigh(S, U1);
                real s = vth * rayleigh(S, U2);
                real cp, sn;
                azimuth(S, &sp, &cp, &sn);
                vr = s * cp; vt = s * sn;
            }
            if (append_particle(S, is_e ? SP_E : SP_CU, 0, j, R_(0), pr, vz, vr, vt, S->id_next++) < 0) return 1;
            if (is_e) { S->emitted_e++; S->charge_cathode += QE * S->c.weight; }
            else S->emitted_cu++;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* one time step: inject -> push -> deposit -> (sort) -> collide + spawn    */
/* -> circuit -> Poisson -> E                                               */
/* ------------------------------------------------------------------ */
int or_step(or_sim* S, int nsteps) {
    for (int s = 0; s < nsteps; ++s) {
        int heavy_step = (S->step % (uint32_t)S->c.heavy_subcycle) == 0;
        if (inject(S)) return 2;
        push_all(S, heavy_step);
        if (S->c.sputter && sputter_emit(S)) return 2;
        deposit_all(S, heavy_step);
        if (collide_all(S, heavy_step)) return 3;
        if (S->c.geom == 0) {
            /* RC circuit: C dV/dt = (V0 - V)/R - I_gap (anode fed through R) */
            S->V += S->c.dt / S->c.C_farad * ((S->c.V0 - S->V) / S->c.R_ohm - S->I_gap);
        }
        if (S->c.field_mode == 1) field_solve(S);
        S->step++;
    }
    return 0;
}

/* initial field from the loaded state (used before the first step) */
int or_prime(or_sim* S) {
    deposit_all(S, 1);
    if (S->c.field_mode == 1) field_solve(S);
    return 0;
}

/* ------------------------------------------------------------------ */
/* getters / diagnostics (Sec. 3, Eq. (21))                                 */
/* ------------------------------------------------------------------ */
int64_t or_count(const or_sim* S) { return S->n; }
uint32_t or_step_index(const or_sim* S) { return S->step; }

static int cmp_u64pair(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* particles sorted by id */
void or_get_particles(const or_sim* S, uint32_t* id, uint8_t* sp, int32_t* iz, int32_t* ir,
                      double* pz, double* pr, double* vz, double* vr, double* vt) {
    uint64_t* k = (uint64_t*)malloc((S->n > 0 ? S->n : 1) * 8);
    for (int64_t p = 0; p < S->n; ++p) k[p] = ((uint64_t)S->id[p] << 32) | (uint64_t)p;
    qsort(k, S->n, 8, cmp_u64pair);
    for (int64_t q = 0; q < S->n; ++q) {
        int64_t p = (int64_t)(k[q] & 0xffffffffu);
        id[q] = S->id[p]; sp[q] = S->sp[p]; iz[q] = S->iz[p]; ir[q] = S->ir[p];
        pz[q] = S->pz[p]; pr[q] = S->pr[p]; vz[q] = S->vz[p]; vr[q] = S->vr[p]; vt[q] = S->vt[p];
    }
    free(k);
}

void or_get_rho(const or_sim* S, int64_t* rho_e, int64_t* rho_h) {
    int64_t nn = (int64_t)S->nzn * S->nrn;
    memcpy(rho_e, S->rho_e, nn * 8);
    memcpy(rho_h, S->rho_h, nn * 8);
}
void or_get_phi(const or_sim* S, double* phi) { memcpy(phi, S->phi, (int64_t)S->nzn * S->nrn * 8); }
void or_get_field(const or_sim* S, double* Ez, double* Er) {
    int64_t nn = (int64_t)S->nzn * S->nrn;
    for (int64_t k = 0; k < nn; ++k) { Ez[k] = S->Ez[k]; Er[k] = S->Er[k]; }
}

/* counters: events[5] of the channels 0-4, nulls, consumed, thr_rej,
 * ratio_viol, iso_fallback, cand_total, emitted_e, emitted_cu,
 * absorbed[3][7], then events of charge exchange, Cu-Cu elastic,
 * Cu2+ -> Cu3+ and Cu3+ -> Cu4+, and the Coulomb pair collisions e-e and
 * e-ion */
void or_get_counters(const or_sim* S, uint64_t* out) {
    int k = 0;
    for (int c = 0; c < CH_CX; ++c) out[k++] = S->events[c];
    out[k++] = S->nulls; out[k++] = S->consumed; out[k++] = S->thr_rej;
    out[k++] = S->ratio_viol; out[k++] = S->iso_fallback; out[k++] = S->cand_total;
    out[k++] = S->emitted_e; out[k++] = S->emitted_cu;
    for (int e = 0; e < 3; ++e) for (int s = 0; s < NSP; ++s) out[k++] = S->absorbed[e][s];
    out[k++] = S->events[CH_CX]; out[k++] = S->events[CH_NN];
    out[k++] = S->events[CH_S3]; out[k++] = S->events[CH_S4];
    out[k++] = S->coul_ee; out[k++] = S->coul_ei;
    out[k++] = S->sput[0]; out[k++] = S->sput[1];
    out[k++] = S->coul_ii;
}

/* scalars: t, V, I_gap, gamma, Qbar, erosion (kg/C), mass ledger (kg),
 * charge ledger (C), sgmax[2], poisson relres, poisson iters, absorbed energy[3] */
void or_get_scalars(const or_sim* S, double* out) {
    uint64_t N[NSP] = {0};
    for (int64_t p = 0; p < S->n; ++p) N[S->sp[p]]++;
    /* Eq. (21) over the heavy species: ionization degree and mean ion charge */
    double ions = 0, qsum = 0;
    for (int s = SP_CUP; s < NSP; ++s) {
        ions += (double)N[s];
        qsum += (double)ZQ[s] * (double)N[s];
    }
    double all = (double)N[SP_CU] + ions;
    double gamma = all > 0 ? ions / all : 0.0;
    double qbar = ions > 0 ? qsum / ions : 0.0;
    double heavy_back = 0;
    for (int s = 1; s < NSP; ++s) heavy_back += (double)S->absorbed[0][s];
    /* net Cu leaving the cathode: injected and sputtered neutrals less the heavies it absorbed */
    double mass = M_CU * S->c.weight * ((double)S->emitted_cu + (double)S->sput[0] - heavy_back);
    double charge = S->charge_cathode;
    out[0] = S->step * S->c.dt;
    out[1] = S->V;
    out[2] = S->I_gap;
    out[3] = gamma;
    out[4] = qbar;
    out[5] = charge != 0 ? mass / charge : 0.0;
    out[6] = mass;
    out[7] = charge;
    out[8] = S->sgmax[0];
    out[9] = S->sgmax[1];
    out[10] = S->poisson_relres;
    out[11] = S->poisson_iters;
    out[12] = S->absorbed_energy[0]; out[13] = S->absorbed_energy[1]; out[14] = S->absorbed_energy[2];
}

/* species density map (m^-3) on the nodes by CIC with the node volumes */
void or_density_map(const or_sim* S, int species, double* out) {
    int64_t nn = (int64_t)S->nzn * S->nrn;
    int64_t* acc = (int64_t*)calloc(nn, 8);
    for (int64_t p = 0; p < S->n; ++p)
        if (S->sp[p] == species) deposit_one(S, acc, S->iz[p], S->ir[p], S->pz[p], S->pr[p], 1);
    for (int i = 0; i < S->nzn; ++i)
        for (int j = 0; j < S->nrn; ++j) {
            int64_t k = (int64_t)i * S->nrn + j;
            out[k] = S->c.weight * (double)acc[k] / 4294967296.0 / node_volume(S, i, j);
        }
    free(acc);
}

/* kinetic-energy spectrum (eV) of one species: counts per bin on [lo, hi) */
void or_energy_spectrum(const or_sim* S, int species, double lo, double hi, int nbins, uint64_t* out) {
    memset(out, 0, nbins * 8);
    for (int64_t p = 0; p < S->n; ++p) {
        if (S->sp[p] != species) continue;
        double e = kinetic(S, p) / QE;
        if (e < lo || e >= hi) continue;
        int b = (int)((e - lo) / (hi - lo) * nbins);
        if (b >= nbins) b = nbins - 1;
        out[b]++;
    }
}

double or_node_volume(const or_sim* S, int i, int j) { return node_volume(S, i, j); }
double or_cell_volume(const or_sim* S, int j) { return cell_volume(S, j); }
int or_real_bytes(void) { return (int)sizeof(real); }
float or_xs_lookup(const or_sim* S, int ch, double eps) { return (float)xs_lookup(S, ch, R_(eps)); }
double or_xs_lookup_d(const or_sim* S, int ch, double eps) { return (double)xs_lookup(S, ch, R_(eps)); }
void or_deposit_weights(double pz, double pr, uint32_t* wz, uint32_t* wr) {
    real a = R_(pz), b = R_(pr);
    *wz = (uint32_t)nearbyint((double)(a * R_(65536)));
    *wr = (uint32_t)nearbyint((double)(b * R_(65536)));
}
