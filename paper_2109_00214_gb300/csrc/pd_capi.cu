// pd_capi.cu -- the C ABI (include/pd.h): workspace layout, constants,
// step orchestration and diagnostics.  Host code; every pipeline step runs
// in the kernels of pd_stream.cu, pd_particles.cu, pd_collide.cu and
// pd_field.cu.
//
// A simulation holds R >= 1 independent runs (an ensemble).  Their cells and
// nodes are laid end to end in one global index space, so that each kernel
// launch advances every run: the sort, scans and candidate machinery see one
// big set of (species, cell) bins; per-particle kernels look up the run of a
// cell and take its constants from a small table.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "pd.h"
#include "pd_field.h"
#include "pd_internal.cuh"
#include "pd_kernels.h"
#include "pd_net.h"

static_assert(PD_NCOUNTERS == pd::NCOUNTERS, "counter layout of the C ABI and the kernels differ");
static_assert(PD_NCH == pd::NCH, "channel count of the C ABI and the kernels differ");

using namespace pd;

namespace {

// CODATA 2018
constexpr double QE = 1.602176634e-19;
constexpr double ME = MASS_E;
constexpr double EPS0_C = 8.8541878128e-12;
constexpr double AMU = AMU_KG;
constexpr double M_CU = MASS_CU;
constexpr double KB = 1.380649e-23;
constexpr double PI = 3.14159265358979323846;
constexpr int ZQ[NSP] = {-1, 0, 1, 2, 2, 3, 4};
constexpr int MAX_RUNS = MAX_RUNS_SMEM;

double species_mass(int s) { return species_mass_kg(s); }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t run_nodes(const pd_config& c) {
    return c.geometry == PD_GEOM_RZ ? (size_t)(c.nz + 1) * (c.nr + 1) : (size_t)c.nz * c.nr;
}

struct Layout {
    size_t total = 0;
    size_t A[7], B[7], M[7];
    size_t count, off, off2, outc, bcnt, act, net, bigq, ovq, ovbits, cntb, mv, mm, partial, nc, nc2, cw, ytab, squeue, cand,
        cand_off, active,
        mid, big, rho_e,
        rho_h, diag, E,
        phi, xsE, xs, ck, ray, hist, spc, state, rs, runs, cell_run, circ, ic, field, wsx, wsy, rmax, grp_base,
        rho_last, rho_prev, rho_prev2, phi_prev, phi_prev2, V_last, V_prev, V_prev2;
    uint32_t nbins_pad, ncell_pad, words_pad, bigq_cap;
    int nsp;                         // species with bins
    uint32_t squeue_cap;             // sputtering impacts per step
    uint64_t cap;                    // physical slots: the configured capacity plus room for the bins' slack
    uint64_t cap_user;               // the configured capacity (particles, live and reserved for spawns)
    uint64_t ncell, nodes, ck_len, rows;
    size_t field_bytes;
};

Layout make_layout(const std::vector<pd_config>& cf) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = align256(o + bytes);
        return r;
    };
    const int R = (int)cf.size();
    uint64_t cap = 0, ncell = 0, nodes = 0, ckl = 0, rows = 0;
    std::vector<int> nz(R), nr(R);
    for (int r = 0; r < R; ++r) {
        cap += (uint64_t)cf[r].capacity;
        ncell += (uint64_t)cf[r].nz * cf[r].nr;
        nodes += run_nodes(cf[r]);
        ckl += (uint64_t)NCLS * cf[r].nr;
        rows += (uint64_t)cf[r].nr;
        nz[r] = cf[r].nz;
        nr[r] = cf[r].nr;
    }
    L.cap_user = cap;
    // slots beyond the capacity hold the slack of the bins: the capacity
    // again, and the four slots per bin that every layout may give a bin
    // whatever its traffic (its three and the rounding up; on a sparse grid
    // the bins outnumber the particles); slot arrays move in groups of four
    // and the mover masks in groups of 128
    const uint64_t nbins_all = ncell * (uint64_t)(cf[0].charge_max >= 3 ? NSP : 5);
    cap = (2 * cap + 4 * nbins_all + 2048 + 127) & ~127ull;
    L.cap = cap;
    L.ncell = ncell;
    L.nodes = nodes;
    L.ck_len = ckl;
    L.rows = rows;
    for (int k = 0; k < 7; ++k) L.A[k] = take(cap * 4);
    for (int k = 0; k < 7; ++k) L.B[k] = take(cap * 4);
    // bins for Cu3+ and Cu4+ only when they can exist
    L.nsp = cf[0].charge_max >= 3 ? NSP : 5;
    L.nbins_pad = scan_padded(ncell * (uint64_t)L.nsp);
    L.ncell_pad = scan_padded(ncell);
    L.words_pad = scan_padded(cap / 32 + 1);
    L.count = take((size_t)L.nbins_pad * 4);               // movers into each bin (cursor of the insertion)
    L.off = take(((size_t)L.nbins_pad + 1) * 4);           // bin starts: the layout, and the next one
    L.off2 = take(((size_t)L.nbins_pad + 1) * 4);
    L.outc = take((size_t)L.nbins_pad * 4);                // particles leaving each bin
    L.bcnt = take((size_t)L.nbins_pad * 4);                // live particles of each bin
    L.act = take((size_t)L.nbins_pad * 4);                 // bin traffic since the last layout
    L.net = take((size_t)L.nbins_pad * 4);
    L.bigq_cap = bigq_max(cap);
    L.bigq = take((size_t)L.bigq_cap * 16);                // long bins with holes
    L.ovq = take((size_t)OVQ_CAP * 4);                     // full bins that borrow slots
    L.ovbits = take(((size_t)L.nbins_pad / 32 + 1) * 4);
    L.cntb = take((size_t)L.nbins_pad * 4);                // re-layout: bin capacities (scan input)
    L.mv = take((size_t)L.words_pad * 4);                  // slots vacated in their bin
    L.mm = take((size_t)L.words_pad * 4);                  // slots whose particle is in the mover records
    for (int k = 0; k < 7; ++k) L.M[k] = take(cap * 4);  // movers at their slots' indices
    const size_t npart = (size_t)std::max(L.nbins_pad, L.ncell_pad) / SCAN_TILE + 1;
    L.partial = take(npart * 4);
    L.nc = take(ncell * 16);                               // candidates of classes 0, 1, 5, 6
    L.nc2 = take(L.nsp == NSP ? ncell * 16 : 16);          // classes 2, 3, 4 (step-wise)
    L.cand = take((size_t)L.ncell_pad * 4);
    L.cand_off = take(((size_t)L.ncell_pad + 1) * 4);
    L.active = take(ncell * 4);
    L.mid = take((size_t)rank_queue_max(cap, RANK_WARP_MAX) * 4);   // id lists queued for rank tables
    L.big = take((size_t)rank_queue_max(cap, RANK_MID_MAX) * 4);
    L.rho_e = take(nodes * 8);
    L.rho_h = take(nodes * 8);
    L.diag = take(nodes * 8);
    L.E = take(nodes * 8);
    L.phi = take(nodes * 8);
    L.xsE = take(XS_N * 4);
    L.xs = take(NCH * XS_N * 4);
    L.ck = take(ckl * 4);
    L.cw = take(2 * rows * 8);                             // W dt / V_cell per row, electron then heavy step
    L.ray = take(1024 * 4);
    L.ytab = take(XS_N * 4);                               // sputtering yield on the table grid
    L.squeue_cap =
        cf[0].sputter ? (uint32_t)std::min<uint64_t>(std::max<uint64_t>(L.cap_user / 16, 4096), 1u << 20) : 16u;
    L.squeue = take((size_t)L.squeue_cap * sizeof(SputRec));
    L.hist = take(4096 * 8);
    L.spc = take((size_t)R * NSP * 8);                     // live particles per run and species
    L.state = take(sizeof(DevState));
    L.rs = take(R * sizeof(RunState));
    L.runs = take(R * sizeof(RunInfo));
    L.cell_run = take(ncell * 2);
    L.circ = take(R * sizeof(RunCircuit));
    L.ic = take(R * sizeof(InjectConsts));
    L.field_bytes = cf[0].field_mode == PD_FIELD_POISSON ? field_workspace_bytes(nz, nr) : 0;
    L.field = take(L.field_bytes);
    L.wsx = take(nodes * 4);                               // warm start: network input and output
    L.wsy = take(nodes * 4);
    L.rmax = take(R * 8);
    L.grp_base = take(R * 4);
    L.rho_last = take(nodes * 8);                          // solve history of the warm start
    L.rho_prev = take(nodes * 8);
    L.rho_prev2 = take(nodes * 8);
    L.phi_prev = take(nodes * 8);
    L.phi_prev2 = take(nodes * 8);
    L.V_last = take(R * 8);
    L.V_prev = take(R * 8);
    L.V_prev2 = take(R * 8);
    L.total = o;
    return L;
}

const char* const KNAMES[PD_NKERNELS] = {"inject",  "push",     "scan_bins", "scatter", "ncand",  "scan_cand",
                                         "collide", "finalize", "poisson",   "efield",  "memset", "other",
                                         "coulomb"};
enum { K_INJECT, K_PUSH, K_SCAN_BINS, K_SCATTER, K_NCAND, K_SCAN_CAND, K_COLLIDE, K_FINALIZE, K_POISSON, K_EFIELD,
       K_MEMSET, K_OTHER, K_COULOMB };

}  // namespace

struct pd_sim {
    std::vector<pd_config> cfgs;
    int R;
    Layout L;
    cudaStream_t stream;
    char* ws;
    int sms;
    Particles A, B;
    uint32_t *count, *off, *off2, *outc, *bcnt, *act, *cntb, *mv, *mm, *partial, *cand, *cand_off, *active, *mid, *big;
    int* net;
    uint4* bigq;
    uint32_t *ovq, *ovbits;
    Particles M;            // movers of the step, at their slots' indices
    bool sorted_valid;      // the bins of A have a layout (after the first step)
    uint4* nc;
    uint4* nc2;
    long long *rho_e, *rho_h, *diag;
    float2* E;
    double* phi;
    float *xsE, *xs, *ck, *ray, *ytab;
    double* cw;
    SputRec* squeue;
    float h_ytab[XS_N];
    unsigned long long *hist, *spc;
    DevState* st;
    RunState* rs;
    RunInfo* runs_dev;
    uint16_t* cell_run;
    RunCircuit* circ_dev;
    InjectConsts* ic_dev;
    std::vector<RunInfo> runs;
    std::vector<uint32_t> node_base;
    FieldSolver field;
    // host copies
    float h_xsE[XS_N];
    float h_xs[NCH][XS_N];
    double eth[NCH];
    CollConsts cc;
    std::vector<InjectConsts> ic;
    float h_ray[1024];
    int64_t step;
    bool primed;
    std::string err;
    // CUDA graph of G steps (G = lcm(2, heavy_subcycle))
    bool graph_on;
    int graph_cycles;
    cudaGraphExec_t gexec;
    int64_t graph_steps;
    uint64_t graph_launches[PD_NKERNELS];
    cudaStream_t capture_stream;
    bool any_inject;
    std::vector<uint16_t> h_cell_run;
    // profiling
    bool prof;
    // diagnosis (environment PD_DEBUG_SYNC=1): the stream is synchronised and
    // the device error bits read after each stage of an eager step; the first
    // failure is reported with the stage's name
    bool debug_sync;
    std::string debug_err;
    struct Rec {
        int k;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    uint64_t launches[PD_NKERNELS];
    pd_tuning tune;
    // warm start of the Poisson solve
    int warm_mode;
    pd_net* warm_net;
    struct Group {
        int B, H, W, first;   // runs of one grid shape; their node bases at grp_base[first ..]
    };
    std::vector<Group> groups;
    float *wsx, *wsy;
    double* rmax;
    uint32_t* grp_base;
    WarmHistory whist;
    int64_t solves;          // Poisson solves since create / load (history depth)
    // species counts of all runs, cached until the particles change
    uint64_t version;        // bumped by every call that changes the particles
    uint64_t spc_version;    // version the cache was taken at (0: none)
    std::vector<unsigned long long> spc_host;
};

namespace {

pd_status fail(pd_sim* s, pd_status code, const std::string& msg) {
    if (s) s->err = msg;
    return code;
}

pd_status cuda_fail(pd_sim* s, cudaError_t e, const char* where) {
    (void)cudaGetLastError();   // reported here: do not leave it to the caller's next CUDA call
    return fail(s, PD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                               \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, #call); \
    } while (0)

// (diagnosis) after a stage: a CUDA error, or device error bits, named by the stage
void debug_stage(pd_sim* s, int k) {
    DevState d;
    cudaError_t e = cudaMemcpyAsync(&d, s->st, sizeof(DevState), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        s->debug_err = std::string("after ") + KNAMES[k] + ": " + cudaGetErrorString(e);
    } else if (d.error) {
        s->debug_err = std::string("after ") + KNAMES[k] + ": device error bits " + std::to_string(d.error) +
                       ", sort checks " + std::to_string(d.sort_fault) + ", step " + std::to_string(s->step);
    }
}

cudaEvent_t take_event(pd_sim* s) {
    if (s->pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    cudaEvent_t e = s->pool.back();
    s->pool.pop_back();
    return e;
}

// launch accounting (`kernels` of the library's kernels the region launches)
// and, when profiling outside graph capture, CUDA events around the region
struct Timed {
    pd_sim* s;
    int k;
    bool capturing;
    cudaEvent_t b;
    Timed(pd_sim* s_, int k_, bool capturing_, int kernels) : s(s_), k(k_), capturing(capturing_), b(nullptr) {
        s->launches[k] += (uint64_t)kernels;
        if (s->prof && !capturing) {
            cudaEvent_t a = take_event(s);
            b = take_event(s);
            cudaEventRecord(a, s->stream);
            s->recs.push_back({k, a, b});
        }
    }
    ~Timed() {
        if (b) cudaEventRecord(b, s->stream);
        if (s->debug_sync && !capturing && s->debug_err.empty()) debug_stage(s, k);
    }
};

KParams kparams(const pd_sim* s, int heavy_step) {
    KParams P;
    const pd_config& c = s->cfgs[0];
    P.geom = c.geometry == PD_GEOM_RZ ? 0 : 1;
    P.nruns = s->R;
    P.ncell = (uint32_t)s->L.ncell;
    P.step = (uint32_t)s->step;
    P.heavy_step = heavy_step;
    P.heavy_coll = s->cfgs[0].heavy_coll;
    P.charge_max = s->cfgs[0].charge_max;
    P.nsp = s->L.nsp;
    P.coulomb = s->cfgs[0].coulomb;
    P.cw_heavy = (uint32_t)s->L.rows;
    P.sputter = s->cfgs[0].sputter;
    P.sput_vth = (float)std::sqrt(KB * s->cfgs[0].sputter_T / M_CU);
    P.xsE = s->xsE;
    P.ytab = s->ytab;
    P.squeue = s->squeue;
    P.squeue_cap = s->L.squeue_cap;
    P.field_on = c.field_mode != PD_FIELD_NONE;
    P.capacity = (unsigned long long)s->L.cap;
    P.user_capacity = (unsigned long long)s->L.cap_user;
    for (int k = 0; k < NSP; ++k) P.masses[k] = species_mass(k);
    P.run0 = s->runs[0];
    P.runs = s->runs_dev;
    P.cell_run = s->cell_run;
    P.rs = s->rs;
    return P;
}

double cell_volume(const pd_config& c, int j) {
    if (c.geometry == PD_GEOM_RZ) return PI * (double)(2 * j + 1) * c.dr * c.dr * c.dz;
    return c.dz * c.dr * c.depth;
}

// Verboncoeur node volumes (linear hat in r); half axial extent on electrodes
double node_volume(const pd_config& c, int i, int j) {
    if (c.geometry != PD_GEOM_RZ) return c.dz * c.dr * c.depth;
    const double dz = c.dz, dr = c.dr;
    const int N = c.nr;
    double v;
    if (j == 0) v = PI * dz * dr * dr / 3.0;
    else if (j == N) v = 2.0 * PI * dz * dr * dr * ((double)N / 2.0 - 1.0 / 6.0);
    else v = 2.0 * PI * dz * dr * dr * (double)j;
    if (i == 0 || i == c.nz) v *= 0.5;
    return v;
}

double mr_class() { return ME * M_CU / (ME + M_CU); }

// NTC majorants from the float tables (see pd_set_cross_section)
void update_collision_consts(pd_sim* s) {
    const double mr = mr_class();
    CollConsts& cc = s->cc;
    cc.kmr = (float)(0.5 * mr / QE);
    cc.kmr_h = (float)(0.5 * (0.5 * M_CU) / QE);
    cc.a_e = (float)(mr / ME);
    cc.a_t = (float)(mr / M_CU);
    for (int ch = 0; ch < NCH; ++ch) cc.kth[ch] = (float)(2.0 * s->eth[ch] * QE / mr);
    cc.di_split_mode = s->cfgs[0].di_split_mode;
    // Coulomb pair factors (q_a q_b)^2 lnL / (8 pi eps0^2 m_ab^2): e-e (m_ab = m_e / 2),
    // then e with Cu+, Cu2+ SW, Cu2+ DI, Cu3+, Cu4+ (m_ab = m_r)
    {
        const double lnl = s->cfgs[0].coulomb_lnl;
        auto kc = [&](int za, int zb, double mab) {
            const double qq = (double)za * (double)zb * QE * QE;
            return qq * qq * lnl / (8.0 * PI * EPS0_C * EPS0_C * mab * mab);
        };
        cc.kc[0] = kc(-1, -1, 0.5 * ME);
        for (int q = 1; q < 6; ++q) cc.kc[q] = kc(-1, ZQ[SP_CUP + q - 1], mr);
        // ion pairs (species a <= b in order), equal masses: m_ab = M / 2
        int cls = 6;
        for (int a = 0; a < 5; ++a)
            for (int b = a; b < 5; ++b) cc.kc[cls++] = kc(ZQ[SP_CUP + a], ZQ[SP_CUP + b], 0.5 * M_CU);
    }
    const int ch0[NCLS] = {CH_EL, CH_SW, CH_S3, CH_S3, CH_S4, CH_CX, CH_NN}, nch[NCLS] = {4, 1, 1, 1, 1, 1, 1};
    for (int k = 0; k < NCLS; ++k) {
        const double kd = (double)(k < NECLS ? cc.kmr : cc.kmr_h);
        double best = 0.0;
        float prev = 0.0f;
        for (int q = 0; q < XS_N; ++q) {
            float sT = 0.0f;
            for (int c = 0; c < nch[k]; ++c) sT = sT + s->h_xs[ch0[k] + c][q];
            if (q > 0) {
                const float smax = sT > prev ? sT : prev;
                const double g = std::sqrt((double)s->h_xsE[q] / kd);
                const double cand = (double)smax * g;
                if (cand > best) best = cand;
            }
            prev = sT;
        }
        best *= 1.0 + 1e-6;
        float f = (float)best;
        if ((double)f < best) f = std::nextafter(f, INFINITY);
        cc.sgmax[k] = f;
    }
}

// per-row factors c_k(j) = W (sigma g)_max dt_coll / V_cell(j) of every run
pd_status upload_ck(pd_sim* s) {
    std::vector<float> ck(s->L.ck_len);
    for (int r = 0; r < s->R; ++r) {
        const pd_config& c = s->cfgs[r];
        const double dtc = c.dt * c.coll_dt_scale;
        const uint32_t base = s->runs[r].ck_base;
        for (int k = 0; k < NECLS; ++k)
            for (int j = 0; j < c.nr; ++j)
                ck[base + (size_t)k * c.nr + j] = (float)(c.weight * (double)s->cc.sgmax[k] * dtc / cell_volume(c, j));
        // heavy pairs collide on heavy steps with the heavy step; (Cu, Cu) pairs
        // number N (N - 1) / 2
        const double dth = dtc * c.heavy_subcycle;
        for (int j = 0; j < c.nr; ++j) {
            ck[base + (size_t)5 * c.nr + j] = (float)(c.weight * (double)s->cc.sgmax[5] * dth / cell_volume(c, j));
            ck[base + (size_t)6 * c.nr + j] =
                (float)(0.5 * c.weight * (double)s->cc.sgmax[6] * dth / cell_volume(c, j));
        }
    }
    // W dt / V_cell(j) per row, with dt_coll and with the heavy step: a
    // cell's density times the time step per particle (Coulomb pairs)
    std::vector<double> cw(2 * s->L.rows);
    for (int r = 0; r < s->R; ++r) {
        const pd_config& c = s->cfgs[r];
        const double dtc = c.dt * c.coll_dt_scale;
        for (int j = 0; j < c.nr; ++j) {
            cw[s->runs[r].row_base + j] = c.weight * dtc / cell_volume(c, j);
            cw[s->L.rows + s->runs[r].row_base + j] = c.weight * (dtc * c.heavy_subcycle) / cell_volume(c, j);
        }
    }
    CK(cudaMemcpyAsync(s->ck, ck.data(), ck.size() * 4, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->cw, cw.data(), cw.size() * 8, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return PD_OK;
}

pd_status read_state(pd_sim* s, DevState* out) {
    CK(cudaMemcpyAsync(out, s->st, sizeof(DevState), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return PD_OK;
}

pd_status check_device_error(pd_sim* s, const DevState& d) {
    if (d.error & ERR_CAPACITY) return fail(s, PD_ERR_CAPACITY, "particle capacity exhausted");
    if (d.error & ERR_IDS) return fail(s, PD_ERR_CAPACITY, "particle id space exhausted");
    if (d.error & ERR_TIMEOUT) return fail(s, PD_ERR_TIMEOUT, "a bounded device wait ran out");
    if (d.error & ERR_NONFINITE) return fail(s, PD_ERR_NONFINITE, "non-finite value in the field solve or a particle's step");
    if (d.error & ERR_BOUNDS) return fail(s, PD_ERR_CAPACITY, "inconsistent slot bookkeeping (reported, not written)");
    return PD_OK;
}

pd_status sync_check(pd_sim* s, DevState* d) {
    pd_status r = read_state(s, d);
    if (r != PD_OK) return r;
    return check_device_error(s, *d);
}

pd_status read_run(pd_sim* s, int run, RunState* out) {
    CK(cudaMemcpyAsync(out, s->rs + run, sizeof(RunState), cudaMemcpyDeviceToHost, s->stream));
    DevState d;
    return sync_check(s, &d);
}

pd_status validate_one(const pd_config* c, std::string& msg) {
    if (!c) { msg = "null config"; return PD_ERR_ARG; }
    if (c->struct_size != sizeof(pd_config) || c->version != PD_CONFIG_VERSION) {
        msg = "pd_config size/version mismatch";
        return PD_ERR_ARG;
    }
    if (c->geometry != PD_GEOM_RZ && c->geometry != PD_GEOM_XY_PERIODIC) { msg = "bad geometry"; return PD_ERR_ARG; }
    if (c->nz < 2 || c->nr < 2 || (int64_t)c->nz * c->nr >= (1 << 24)) { msg = "grid must be >= 2x2 and < 2^24 cells"; return PD_ERR_ARG; }
    if (!(c->dz > 0) || !(c->dr > 0) || !(c->dt > 0) || !(c->weight > 0)) { msg = "dz, dr, dt, weight must be > 0"; return PD_ERR_ARG; }
    if (c->geometry == PD_GEOM_XY_PERIODIC && !(c->depth > 0)) { msg = "depth must be > 0"; return PD_ERR_ARG; }
    if (c->heavy_subcycle < 1) { msg = "heavy_subcycle must be >= 1"; return PD_ERR_ARG; }
    if (c->capacity < 1 || c->capacity > 0xFFFFFFFFll) { msg = "capacity must be in [1, 2^32)"; return PD_ERR_ARG; }
    if (c->field_mode < 0 || c->field_mode > 2) { msg = "bad field_mode"; return PD_ERR_ARG; }
    if (c->field_mode == PD_FIELD_POISSON && c->geometry != PD_GEOM_RZ) { msg = "Poisson field needs r-z"; return PD_ERR_ARG; }
    if (c->field_mode == PD_FIELD_POISSON && !field_grid_ok(c->nz, c->nr)) { msg = "Poisson multigrid needs nz, nr = m * 2^k with m <= 8"; return PD_ERR_ARG; }
    if (!(c->coll_dt_scale >= 0)) { msg = "coll_dt_scale must be >= 0"; return PD_ERR_ARG; }
    if (c->heavy_coll != 0 && c->heavy_coll != 1) { msg = "heavy_coll must be 0 or 1"; return PD_ERR_ARG; }
    if (c->charge_max < 2 || c->charge_max > 4) { msg = "charge_max must be 2, 3 or 4"; return PD_ERR_ARG; }
    if (c->coulomb != 0 && c->coulomb != 1) { msg = "coulomb must be 0 or 1"; return PD_ERR_ARG; }
    if (c->sputter != 0 && c->sputter != 1) { msg = "sputter must be 0 or 1"; return PD_ERR_ARG; }
    if (c->reserved1 != 0) { msg = "reserved1 must be 0"; return PD_ERR_ARG; }
    if (c->sputter && !(c->sputter_T > 0.0 && std::isfinite(c->sputter_T))) {
        msg = "sputter_T must be positive";
        return PD_ERR_ARG;
    }
    if (c->coulomb && !(c->coulomb_lnl > 0.0 && std::isfinite(c->coulomb_lnl))) {
        msg = "coulomb_lnl must be positive";
        return PD_ERR_ARG;
    }
    if (c->geometry == PD_GEOM_RZ && c->inject_on) {
        if (!(c->tip_radius > 0) || c->tip_radius / c->dr > 63) { msg = "tip must span 1..63 cells"; return PD_ERR_ARG; }
    }
    return PD_OK;
}

// runs of one simulation share everything that is not per-run geometry,
// weight, seed, circuit or emission
pd_status validate(const pd_config* cfgs, int n, std::string& msg) {
    if (!cfgs || n < 1 || n > MAX_RUNS) { msg = "need 1.." + std::to_string(MAX_RUNS) + " runs"; return PD_ERR_ARG; }
    uint64_t cells = 0, cap = 0;
    for (int r = 0; r < n; ++r) {
        pd_status e = validate_one(&cfgs[r], msg);
        if (e != PD_OK) return e;
        const pd_config &a = cfgs[0], &b = cfgs[r];
        if (b.geometry != a.geometry || b.dt != a.dt || b.heavy_subcycle != a.heavy_subcycle ||
            b.field_mode != a.field_mode || b.coll_dt_scale != a.coll_dt_scale || b.di_on != a.di_on ||
            b.di_split_mode != a.di_split_mode || b.heavy_coll != a.heavy_coll || b.charge_max != a.charge_max ||
            b.coulomb != a.coulomb || b.coulomb_lnl != a.coulomb_lnl || b.sputter != a.sputter ||
            b.sputter_T != a.sputter_T) {
            msg = "runs differ in geometry, dt, heavy_subcycle, field_mode, coll_dt_scale, double-ionization "
                  "or heavy-collision settings";
            return PD_ERR_ARG;
        }
        cells += (uint64_t)b.nz * b.nr;
        cap += (uint64_t)b.capacity;
    }
    if (cells >= (1u << 24)) { msg = "all runs together must have < 2^24 cells"; return PD_ERR_ARG; }
    // the slot arrays hold the capacity twice (the bins' slack) and four slots per bin
    if (2 * cap + 28 * cells + 4096 > 0xFFFFFFF0ull) {
        msg = "all runs together must have a capacity below 2^31 particles";
        return PD_ERR_ARG;
    }
    return PD_OK;
}

InjectConsts make_injection(const pd_config& c) {
    InjectConsts ic;
    std::memset(&ic, 0, sizeof(ic));
    if (c.geometry != PD_GEOM_RZ || !c.inject_on) return ic;
    const double dr = c.dr, rt = c.tip_radius;
    const float rtip_cells = (float)(rt / dr);
    int n = 0;
    for (int j = 0; (double)j * dr < rt && j < c.nr && j < 64; ++j) {
        const double rhi = std::fmin((j + 1) * dr, rt), rlo = j * dr;
        ic.area[j] = PI * (rhi * rhi - rlo * rlo);
        ic.lo[j] = (float)j;
        ic.hi[j] = (j + 1) * dr <= rt ? (float)(j + 1) : rtip_cells;
        n = j + 1;
    }
    ic.ntip = n;
    ic.dt = c.dt;
    ic.weight = c.weight;
    ic.beta = c.beta;
    ic.work = c.work_function;
    ic.ratio = c.neutral_ratio;
    ic.vth = (float)std::sqrt(KB * c.neutral_T / M_CU);
    return ic;
}

int grid_for(pd_sim* s, int per_sm) { return s->sms * per_sm; }

pd_tuning default_tuning() {
    pd_tuning t;
    t.push_blocks_per_sm = 8;
    t.bincount_blocks_per_sm = 8;
    t.scatter_blocks_per_sm = 8;
    t.ncand_blocks_per_sm = 8;
    t.collide_blocks_per_sm = 16;
    t.mg_threads = 256;
    t.mg_max_blocks = 1216;
    return t;
}

bool tuning_ok(const pd_tuning& t) {
    auto bps = [](int v) { return v >= 1 && v <= 64; };
    return bps(t.push_blocks_per_sm) && bps(t.bincount_blocks_per_sm) && bps(t.scatter_blocks_per_sm) &&
           bps(t.ncand_blocks_per_sm) && bps(t.collide_blocks_per_sm) && t.mg_threads >= 64 &&
           t.mg_threads <= 1024 && t.mg_threads % 32 == 0 && t.mg_max_blocks >= 1 && t.mg_max_blocks <= 65535;
}

void apply_tuning(pd_sim* s, const pd_tuning& t) {
    s->tune = t;
    s->field.threads = t.mg_threads;
    s->field.max_blocks = t.mg_max_blocks;
}

size_t total_nodes(const pd_sim* s) { return (size_t)s->L.nodes; }

// before each Poisson solve: the solve history, then the starting point
// (PD_WARM_PREVIOUS: phi as it is; PD_WARM_EXTRAPOLATE: set with the history
// shift once two solutions exist)
pd_status warm_start(pd_sim* s, int* kernels) {
    const bool extrapolate = s->warm_mode == PD_WARM_EXTRAPOLATE && s->solves >= 2;
    warm_history(s->field, s->rho_e, s->rho_h, s->runs_dev, s->rs, s->phi, s->whist, extrapolate, s->stream);
    *kernels += 1;
    // the learned forms need one (delta) or two (extrapolated) earlier
    // solves; until then the previous potential stands
    int form = -1;
    if (s->warm_mode == PD_WARM_LEARNED) form = WARM_ABSOLUTE;
    else if (s->warm_mode == PD_WARM_LEARNED_DELTA && s->solves >= 1) form = WARM_DELTA;
    else if (s->warm_mode == PD_WARM_LEARNED_EXTRAP && s->solves >= 2) form = WARM_EXTRAP;
    if (s->warm_mode == PD_WARM_COLD) {
        warm_apply(s->field, nullptr, s->whist, WARM_ABSOLUTE, s->runs_dev, s->rs, s->rmax, s->phi, s->stream);
        *kernels += 1;
    } else if (form >= 0) {
        warm_inputs(s->field, s->whist, form, s->runs_dev, s->rmax, s->wsx, s->stream);
        for (const auto& g : s->groups)
            if (net_forward_at(s->warm_net, s->wsx, s->wsy, g.B, g.H, g.W, s->grp_base + g.first,
                               (int64_t)total_nodes(s), s->stream))
                return PD_ERR_CUDA;
        warm_apply(s->field, s->wsy, s->whist, form, s->runs_dev, s->rs, s->rmax, s->phi, s->stream);
        *kernels += 3 + 6 * (int)s->groups.size();   // rmax, x, apply; six layers per group
    }
    s->solves += 1;
    return cudaGetLastError() == cudaSuccess ? PD_OK : PD_ERR_CUDA;
}

pd_status prime(pd_sim* s) {
    KParams P = kparams(s, 1);
    CK(cudaMemsetAsync(s->rho_e, 0, total_nodes(s) * 8, s->stream));
    CK(cudaMemsetAsync(s->rho_h, 0, total_nodes(s) * 8, s->stream));
    {
        Timed t(s, K_OTHER, false, 1);
        launch_deposit(s->A, s->rho_e, s->rho_h, s->st, P, grid_for(s, 8), s->stream);
    }
    if (s->cfgs[0].field_mode == PD_FIELD_POISSON) {
        Timed t(s, K_POISSON, false, 2);   // + the warm start's and the solve's kernels, counted below
        int nk = 0;
        if (warm_start(s, &nk) != PD_OK) return fail(s, PD_ERR_CUDA, "warm start failed");
        const cudaError_t fe = field_solve(s->field, s->rho_e, s->rho_h, s->phi, s->E, s->runs_dev, s->rs, 1, 0,
                                           s->stream, &nk);
        if (fe != cudaSuccess) return cuda_fail(s, fe, "field solve");
        s->launches[K_POISSON] += (uint64_t)nk;
        field_efield(s->field, s->phi, s->runs_dev, s->E, s->st, s->rs, s->stream);
    }
    CK(cudaGetLastError());
    s->primed = true;
    return PD_OK;
}

// one electron step, issued on the stream; `capturing` when recorded into a graph
pd_status issue_step(pd_sim* s, bool capturing) {
    const pd_config& c = s->cfgs[0];
    const int heavy = (s->step % c.heavy_subcycle) == 0;
    const KParams P = kparams(s, heavy);
    const uint32_t nbins = (uint32_t)s->L.ncell * (uint32_t)s->L.nsp;
    const int gpart = grid_for(s, s->tune.push_blocks_per_sm);
    const size_t nodes = total_nodes(s);
    if (s->any_inject) {
        Timed t(s, K_INJECT, capturing, 1);
        launch_inject(s->A, s->E, s->st, P, s->ic_dev, s->ray, s->stream);
    }
    {
        Timed t(s, K_MEMSET, capturing, 0);   // memsets, no kernels
        cudaMemsetAsync(s->rho_e, 0, nodes * 8, s->stream);
        if (heavy) cudaMemsetAsync(s->rho_h, 0, nodes * 8, s->stream);
        // vacated-slot and mover bits are OR-ed in by the push: start from zero
        cudaMemsetAsync(s->mv, 0, (size_t)s->L.words_pad * 4, s->stream);
        cudaMemsetAsync(s->mm, 0, (size_t)s->L.words_pad * 4, s->stream);
    }
    {
        Timed t(s, K_PUSH, capturing, 1);
        launch_push(s->A, s->E, s->rho_e, s->rho_h, s->outc, s->count, s->mv, s->mm, s->M, s->st, P, gpart,
                    s->stream);
    }
    if (c.sputter && heavy && c.geometry == PD_GEOM_RZ) {
        // ions reach the electrodes on heavy steps: their sputtered atoms join this step's sort
        Timed t(s, K_INJECT, capturing, 1);
        launch_sputter(s->M, s->mm, s->st, P, s->ray, s->count, s->stream);
    }
    {
        SortArgs a;
        a.A = s->A;
        a.B = s->B;
        a.M = s->M;
        a.mv = s->mv;
        a.mm = s->mm;
        a.off = s->off;
        a.off2 = s->off2;
        a.cnt = s->bcnt;
        a.out_cnt = s->outc;
        a.in_cnt = s->count;
        a.cap = s->cntb;
        a.act = s->act;
        a.net = s->net;
        a.bigq = s->bigq;
        a.bigq_cap = s->L.bigq_cap;
        a.ovq = s->ovq;
        a.ovbits = s->ovbits;
        a.partial = s->partial;
        a.nbins = nbins;
        a.nbins_pad = s->L.nbins_pad;
        a.slots = s->L.cap;
        a.ncell_pad = s->L.ncell_pad;
        {
            // heavy bins: counts, holes closed, slots borrowed (k_bins, k_compact_big, k_borrow)
            Timed t(s, K_SCATTER, capturing, 3);
            launch_sort(a, s->st, P, s->sms, s->stream);
        }
        {
            // the re-layout of the heavy bins (three kernels, a scan of three,
            // and four more) returns at once unless a heavy bin overflowed
            Timed t(s, K_SCAN_BINS, capturing, 10);
            launch_relayout(a, s->st, P, grid_for(s, s->tune.bincount_blocks_per_sm),
                            grid_for(s, s->tune.scatter_blocks_per_sm), s->stream, !s->sorted_valid);
        }
        {
            // electron bins laid out (a scan of three, k_ebins), movers
            // inserted (k_insert, k_insert_dense)
            Timed t(s, K_SCATTER, capturing, 6);
            launch_insert(a, s->st, P, grid_for(s, s->tune.scatter_blocks_per_sm), s->stream);
        }
    }
    s->sorted_valid = true;
    {
        Timed t(s, K_NCAND, capturing, 1);
        launch_ncand(s->bcnt, s->ck, s->nc, s->nc2, s->cand, s->active, s->mid, s->big, s->st, P,
                     grid_for(s, s->tune.ncand_blocks_per_sm), s->stream);
    }
    {
        Timed t(s, K_SCAN_CAND, capturing, 3);
        launch_scan(s->cand, s->cand_off, s->partial, s->L.ncell_pad, s->stream);
    }
    {
        Timed t(s, K_COLLIDE, capturing, 3);
        launch_collide(s->A, s->B, s->off, s->bcnt, s->nc, s->nc2, s->cand_off, s->active, s->mid, s->big, s->st,
                       s->rho_e, s->rho_h,
                       s->xsE, s->xs, s->cw, P, s->cc, nbins, s->sms, grid_for(s, s->tune.collide_blocks_per_sm),
                       s->stream);
    }
    if (P.coulomb) {
        Timed t(s, K_COULOMB, capturing, 1);
        launch_coulomb(s->A, s->B, s->off, s->bcnt, s->st, P, s->cc, s->cw, s->sms, s->stream);
    }
    {
        Timed t(s, K_FINALIZE, capturing, 1);
        launch_finalize(s->off, nbins, s->cand_off, s->st, P, s->circ_dev, c.dt, c.geometry == PD_GEOM_RZ, s->stream);
    }
    if (c.field_mode == PD_FIELD_POISSON) {
        {
            Timed t(s, K_POISSON, capturing, 0);
            int nk = 0;
            if (warm_start(s, &nk) != PD_OK) return fail(s, PD_ERR_CUDA, "warm start failed");
            const bool host_check = !capturing && !s->graph_on;
            const cudaError_t fe = field_solve(s->field, s->rho_e, s->rho_h, s->phi, s->E, s->runs_dev, s->rs,
                                               host_check ? 1 : 0, s->graph_cycles, s->stream, &nk);
            if (fe != cudaSuccess) return cuda_fail(s, fe, "field solve");
            s->launches[K_POISSON] += (uint64_t)nk;
        }
        {
            Timed t(s, K_EFIELD, capturing, 2);
            field_efield(s->field, s->phi, s->runs_dev, s->E, s->st, s->rs, s->stream);
        }
    }
    s->step += 1;
    if (!s->debug_err.empty()) return fail(s, PD_ERR_CUDA, "PD_DEBUG_SYNC: " + s->debug_err);
    return PD_OK;
}

int graph_period(const pd_sim* s) {
    const int h = s->cfgs[0].heavy_subcycle;
    return (h % 2 == 0) ? h : 2 * h;   // whole heavy cycles, even
}

// ---- checkpoint file: a header, then the sections in a fixed order ----
constexpr char CKPT_MAGIC[8] = {'P', 'D', 'C', 'K', 'P', 'T', '0', '1'};
constexpr uint32_t CKPT_VERSION = 4;

struct CkptHeader {
    char magic[8];
    uint32_t version, nruns;
    uint32_t cfg_size, runstate_size, devstate_size, sorted_valid;
    uint32_t primed, pad0;
    int64_t step;
    uint64_t n_slots, n_off, nodes, cap;
};

bool same_config(const pd_config& a, const pd_config& b) {
    return a.struct_size == b.struct_size && a.version == b.version && a.geometry == b.geometry && a.nz == b.nz &&
           a.nr == b.nr && a.dz == b.dz && a.dr == b.dr && a.depth == b.depth && a.dt == b.dt &&
           a.heavy_subcycle == b.heavy_subcycle && a.weight == b.weight && a.seed == b.seed && a.run == b.run &&
           a.field_mode == b.field_mode && a.inject_on == b.inject_on && a.di_on == b.di_on &&
           a.di_split_mode == b.di_split_mode && a.coll_dt_scale == b.coll_dt_scale && a.V0 == b.V0 &&
           a.R_ohm == b.R_ohm && a.C_farad == b.C_farad && a.beta == b.beta && a.tip_radius == b.tip_radius &&
           a.work_function == b.work_function && a.neutral_ratio == b.neutral_ratio &&
           a.neutral_T == b.neutral_T && a.poisson_tol == b.poisson_tol &&
           a.poisson_max_cycles == b.poisson_max_cycles && a.heavy_coll == b.heavy_coll &&
           a.charge_max == b.charge_max && a.coulomb == b.coulomb && a.coulomb_lnl == b.coulomb_lnl &&
           a.sputter == b.sputter && a.sputter_T == b.sputter_T && a.capacity == b.capacity;
}

struct File {
    std::FILE* f;
    explicit File(std::FILE* f_) : f(f_) {}
    ~File() {
        if (f) std::fclose(f);
    }
    bool put(const void* p, size_t n) { return n == 0 || std::fwrite(p, 1, n, f) == n; }
    bool get(void* p, size_t n) { return n == 0 || std::fread(p, 1, n, f) == n; }
};

// device range <-> file through a bounded host buffer
pd_status dev_to_file(pd_sim* s, File& F, const void* dev, size_t bytes) {
    std::vector<char> h(std::min<size_t>(bytes, (size_t)64 << 20));
    for (size_t o = 0; o < bytes; o += h.size()) {
        const size_t n = std::min(h.size(), bytes - o);
        CK(cudaMemcpyAsync(h.data(), (const char*)dev + o, n, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        if (!F.put(h.data(), n)) return fail(s, PD_ERR_ARG, "checkpoint write failed");
    }
    return PD_OK;
}

pd_status file_to_dev(pd_sim* s, File& F, void* dev, size_t bytes) {
    std::vector<char> h(std::min<size_t>(bytes, (size_t)64 << 20));
    for (size_t o = 0; o < bytes; o += h.size()) {
        const size_t n = std::min(h.size(), bytes - o);
        if (!F.get(h.data(), n)) return fail(s, PD_ERR_ARG, "checkpoint file is truncated");
        CK(cudaMemcpyAsync((char*)dev + o, h.data(), n, cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    return PD_OK;
}

void fill_event_pool(pd_sim* s) {
    if (!s->pool.empty() || !s->recs.empty()) return;
    for (int k = 0; k < 8192; ++k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) break;
        s->pool.push_back(e);
    }
}

// synchronise, add the recorded kernel times per kernel id into ms (may be
// null) and return the events to the pool
pd_status collect_profile(pd_sim* s, double* ms) {
    CK(cudaStreamSynchronize(s->stream));
    if (ms)
        for (int k = 0; k < PD_NKERNELS; ++k) ms[k] = 0.0;
    for (auto& r : s->recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess && ms) ms[r.k] += t;
        s->pool.push_back(r.a);
        s->pool.push_back(r.b);
    }
    s->recs.clear();
    return PD_OK;
}

pd_status drop_graph(pd_sim* s) {
    if (s->gexec) {
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
    }
    return PD_OK;
}

// capture G steps into one executable graph (the first step of the capture
// must be a multiple of G and the sorted order must already exist)
pd_status build_graph(pd_sim* s) {
    drop_graph(s);
    const int G = graph_period(s);
    cudaGraph_t g = nullptr;
    uint64_t before[PD_NKERNELS];
    std::memcpy(before, s->launches, sizeof(before));
    // record on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the caller's
    if (!s->capture_stream) CK(cudaStreamCreateWithFlags(&s->capture_stream, cudaStreamNonBlocking));
    CK(cudaStreamSynchronize(s->stream));
    cudaStream_t user = s->stream;
    s->stream = s->capture_stream;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        s->stream = user;
        return cuda_fail(s, e, "cudaStreamBeginCapture");
    }
    const int64_t step0 = s->step;
    pd_status r = PD_OK;
    for (int k = 0; k < G && r == PD_OK; ++k) r = issue_step(s, true);
    e = cudaStreamEndCapture(s->stream, &g);
    s->stream = user;
    s->step = step0;           // capture only recorded the steps
    for (int k = 0; k < PD_NKERNELS; ++k) {   // launches of one replay
        s->graph_launches[k] = s->launches[k] - before[k];
        s->launches[k] = before[k];
    }
    if (r != PD_OK) return r;
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&s->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaGraphInstantiate");
    s->graph_steps = G;
    return PD_OK;
}

pd_status create_common(const pd_config* cfgs, int n, void* ws, size_t bytes, void* stream, pd_sim** out) {
    if (!out) return PD_ERR_ARG;
    *out = nullptr;
    std::string msg;
    pd_status v = validate(cfgs, n, msg);
    if (v != PD_OK) {
        std::fprintf(stderr, "pd_create: %s\n", msg.c_str());
        return v;
    }
    std::vector<pd_config> cf(cfgs, cfgs + n);
    Layout L = make_layout(cf);
    if (!ws || bytes < L.total || ((uintptr_t)ws & 255)) return PD_ERR_ARG;
    pd_sim* s = new (std::nothrow) pd_sim();
    if (!s) return PD_ERR_ARG;
    s->cfgs = cf;
    s->R = n;
    s->L = L;
    s->stream = (cudaStream_t)stream;
    s->ws = (char*)ws;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = collide_setup();
    if (e != cudaSuccess) {
        delete s;
        return PD_ERR_CUDA;
    }
    char* w = s->ws;
    auto P32 = [&](size_t o) { return (uint32_t*)(w + o); };
    auto PF = [&](size_t o) { return (float*)(w + o); };
    s->A = Particles{P32(L.A[0]), PF(L.A[1]), PF(L.A[2]), PF(L.A[3]), PF(L.A[4]), PF(L.A[5]), P32(L.A[6])};
    s->B = Particles{P32(L.B[0]), PF(L.B[1]), PF(L.B[2]), PF(L.B[3]), PF(L.B[4]), PF(L.B[5]), P32(L.B[6])};
    s->count = P32(L.count);
    s->off = P32(L.off);
    s->off2 = P32(L.off2);
    s->outc = P32(L.outc);
    s->bcnt = P32(L.bcnt);
    s->act = P32(L.act);
    s->net = (int*)(w + L.net);
    s->bigq = (uint4*)(w + L.bigq);
    s->ovq = P32(L.ovq);
    s->ovbits = P32(L.ovbits);
    s->cntb = P32(L.cntb);
    s->mv = P32(L.mv);
    s->mm = P32(L.mm);
    s->M = Particles{P32(L.M[0]), PF(L.M[1]), PF(L.M[2]), PF(L.M[3]), PF(L.M[4]), PF(L.M[5]), P32(L.M[6])};
    s->sorted_valid = false;
    s->partial = P32(L.partial);
    s->nc = (uint4*)(w + L.nc);
    s->nc2 = (uint4*)(w + L.nc2);
    s->cand = P32(L.cand);
    s->cand_off = P32(L.cand_off);
    s->active = P32(L.active);
    s->mid = P32(L.mid);
    s->big = P32(L.big);
    s->rho_e = (long long*)(w + L.rho_e);
    s->rho_h = (long long*)(w + L.rho_h);
    s->diag = (long long*)(w + L.diag);
    s->E = (float2*)(w + L.E);
    s->phi = (double*)(w + L.phi);
    s->xsE = PF(L.xsE);
    s->xs = PF(L.xs);
    s->ck = PF(L.ck);
    s->cw = (double*)(w + L.cw);
    s->ray = PF(L.ray);
    s->ytab = PF(L.ytab);
    s->squeue = (SputRec*)(w + L.squeue);
    s->hist = (unsigned long long*)(w + L.hist);
    s->spc = (unsigned long long*)(w + L.spc);
    s->st = (DevState*)(w + L.state);
    s->rs = (RunState*)(w + L.rs);
    s->runs_dev = (RunInfo*)(w + L.runs);
    s->cell_run = (uint16_t*)(w + L.cell_run);
    s->circ_dev = (RunCircuit*)(w + L.circ);
    s->ic_dev = (InjectConsts*)(w + L.ic);
    s->wsx = PF(L.wsx);
    s->wsy = PF(L.wsy);
    s->rmax = (double*)(w + L.rmax);
    s->grp_base = P32(L.grp_base);
    s->warm_mode = PD_WARM_PREVIOUS;
    s->warm_net = nullptr;
    s->version = 1;
    s->spc_version = 0;
    s->whist = WarmHistory{(double*)(w + L.rho_last), (double*)(w + L.rho_prev), (double*)(w + L.rho_prev2),
                          (double*)(w + L.phi_prev), (double*)(w + L.phi_prev2), (double*)(w + L.V_last),
                          (double*)(w + L.V_prev), (double*)(w + L.V_prev2)};
    s->solves = 0;
    for (int k = 0; k < XS_N; ++k) {
        const int ex = XS_EMIN_EXP + k / XS_SUB, j = k % XS_SUB;
        s->h_xsE[k] = (float)std::ldexp(1.0 + (double)j / XS_SUB, ex);
    }
    std::memset(s->h_xs, 0, sizeof(s->h_xs));
    std::memset(s->h_ytab, 0, sizeof(s->h_ytab));
    for (int k = 0; k < NCH; ++k) s->eth[k] = 0.0;
    update_collision_consts(s);
    for (int k = 0; k < 1024; ++k) s->h_ray[k] = (float)std::sqrt(-2.0 * std::log(1.0 - (double)k / 1024.0));
    // run tables
    s->runs.resize(n);
    s->node_base.resize(n);
    std::vector<RunCircuit> circ(n);
    std::vector<uint16_t> cell_run(L.ncell);
    std::vector<RunState> rs(n);
    s->ic.resize(n);
    uint32_t cb = 0, nb = 0, kb = 0, rb = 0;
    for (int r = 0; r < n; ++r) {
        const pd_config& c = cf[r];
        RunInfo& RI = s->runs[r];
        std::memset(&RI, 0, sizeof(RI));
        RI.nz = c.nz;
        RI.nr = c.nr;
        RI.nzn = c.geometry == PD_GEOM_RZ ? c.nz + 1 : c.nz;
        RI.nrn = c.geometry == PD_GEOM_RZ ? c.nr + 1 : c.nr;
        RI.inv_nr = 1.0f / (float)c.nr;
        RI.cell_base = cb;
        RI.node_base = nb;
        RI.ncell = (uint32_t)c.nz * (uint32_t)c.nr;
        RI.seed = c.seed;
        RI.run = c.run;
        RI.ck_base = kb;
        RI.row_base = rb;
        const double dte = c.dt, dth = c.dt * c.heavy_subcycle;
        for (int sp = 0; sp < NSP; ++sp) {
            const double dts = sp == SP_E ? dte : dth;
            RI.qmdt[sp] = (float)((double)ZQ[sp] * QE / species_mass(sp) * dts);
            RI.dtz[sp] = (float)(dts / c.dz);
            RI.dtr[sp] = (float)(dts / c.dr);
        }
        RI.weight = c.weight;
        for (uint32_t q = 0; q < RI.ncell; ++q) cell_run[cb + q] = (uint16_t)r;
        s->node_base[r] = nb;
        cb += RI.ncell;
        nb += (uint32_t)run_nodes(c);
        kb += (uint32_t)NCLS * (uint32_t)c.nr;
        rb += (uint32_t)c.nr;
        circ[r] = RunCircuit{c.V0, c.R_ohm, c.C_farad};
        std::memset(&rs[r], 0, sizeof(RunState));
        rs[r].V = c.V0;
        s->ic[r] = make_injection(c);
    }
    s->any_inject = false;
    for (int r = 0; r < n; ++r) s->any_inject = s->any_inject || s->ic[r].ntip > 0;
    s->h_cell_run = cell_run;
    std::memset(s->graph_launches, 0, sizeof(s->graph_launches));
    s->step = 0;
    s->primed = false;
    s->prof = false;
    {
        const char* d = std::getenv("PD_DEBUG_SYNC");
        s->debug_sync = d && d[0] == '1';
    }
    s->graph_on = false;
    s->graph_cycles = 4;
    s->tune = default_tuning();
    s->gexec = nullptr;
    s->capture_stream = nullptr;
    s->graph_steps = 0;
    std::memset(s->launches, 0, sizeof(s->launches));
    // zero everything but the two particle buffers
    const size_t z0 = L.count;
    e = cudaMemsetAsync(w + z0, 0, L.total - z0, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->xsE, s->h_xsE, sizeof(s->h_xsE), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->ray, s->h_ray, sizeof(s->h_ray), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->runs_dev, s->runs.data(), n * sizeof(RunInfo), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->cell_run, cell_run.data(), cell_run.size() * 2, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->circ_dev, circ.data(), n * sizeof(RunCircuit), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->rs, rs.data(), n * sizeof(RunState), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->ic_dev, s->ic.data(), n * sizeof(InjectConsts), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "pd_create: %s\n", cudaGetErrorString(e));
        delete s;
        return PD_ERR_CUDA;
    }
    if (cf[0].field_mode == PD_FIELD_POISSON) {
        if (field_init(s->field, cf, s->node_base, s->phi, w + L.field, L.field_bytes, s->stream) != 0) {
            field_free(s->field);
            delete s;
            return PD_ERR_CUDA;
        }
    }
    pd_status ur = upload_ck(s);
    if (ur != PD_OK) {
        field_free(s->field);
        delete s;
        return ur;
    }
    *out = s;
    return PD_OK;
}

pd_status load_device(pd_sim* s, int run, int64_t n, const uint8_t* sp, const int32_t* iz, const int32_t* ir,
                      const float* pz, const float* pr, const float* vz, const float* vr, const float* vt);

// host arrays: copied straight to the device (fast from pinned memory) --
// positions and velocities into their slots, species and cell indices into
// the other particle buffer, free between steps -- and checked and packed
// there by the device load

// particles in bins plus the tail's slots (loaded or spawned, not yet
// sorted) plus n more: above the configured capacity?
bool load_exceeds(const pd_sim* s, const DevState& d, int64_t n) {
    return d.n_live + d.n_e + (d.n_slots - d.tail_base) + (uint64_t)n > s->L.cap_user;
}

pd_status load_host(pd_sim* s, int run, int64_t n, const uint8_t* sp, const int32_t* iz, const int32_t* ir,
                    const float* pz, const float* pr, const float* vz, const float* vr, const float* vt) {
    if (!s) return PD_ERR_ARG;
    ++s->version;
    if (run < 0 || run >= s->R) return fail(s, PD_ERR_ARG, "bad run index");
    if (n < 0) return fail(s, PD_ERR_ARG, "n < 0");
    if (n == 0) return PD_OK;
    DevState d;
    pd_status r = sync_check(s, &d);
    if (r != PD_OK) return r;
    if (d.n_slots + (uint64_t)n > s->L.cap || load_exceeds(s, d, n))
        return fail(s, PD_ERR_CAPACITY, "load exceeds capacity");
    const size_t o = d.n_slots, nb = (size_t)n * 4;
    int32_t* diz = reinterpret_cast<int32_t*>(s->B.key + o);
    int32_t* dir = reinterpret_cast<int32_t*>(s->B.id + o);
    uint8_t* dsp = reinterpret_cast<uint8_t*>(s->B.pz + o);
    CK(cudaMemcpyAsync(diz, iz, nb, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(dir, ir, nb, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(dsp, sp, (size_t)n, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->A.pz + o, pz, nb, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->A.pr + o, pr, nb, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->A.vz + o, vz, nb, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->A.vr + o, vr, nb, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->A.vt + o, vt, nb, cudaMemcpyHostToDevice, s->stream));
    return load_device(s, run, n, dsp, diz, dir, s->A.pz + o, s->A.pr + o, s->A.vz + o, s->A.vr + o, s->A.vt + o);
}

pd_status load_device(pd_sim* s, int run, int64_t n, const uint8_t* sp, const int32_t* iz, const int32_t* ir,
                      const float* pz, const float* pr, const float* vz, const float* vr, const float* vt) {
    if (!s) return PD_ERR_ARG;
    ++s->version;
    if (run < 0 || run >= s->R) return fail(s, PD_ERR_ARG, "bad run index");
    if (n < 0) return fail(s, PD_ERR_ARG, "n < 0");
    if (n == 0) return PD_OK;
    DevState d;
    pd_status r = sync_check(s, &d);
    if (r != PD_OK) return r;
    RunState rs;
    r = read_run(s, run, &rs);
    if (r != PD_OK) return r;
    if (d.n_slots + (uint64_t)n > s->L.cap || load_exceeds(s, d, n))
        return fail(s, PD_ERR_CAPACITY, "load exceeds capacity");
    if ((uint64_t)rs.id_next + (uint64_t)n > 0xFFFFFFFFull) return fail(s, PD_ERR_CAPACITY, "id space exhausted");
    const RunInfo& RI = s->runs[run];
    const size_t o = d.n_slots;
    unsigned int bad = 0;
    unsigned int* dbad = &s->st->load_bad;
    CK(cudaMemsetAsync(dbad, 0, 4, s->stream));
    // species codes up to the configured highest charge (Cu2+ DI is 4, Cu3+ 5, Cu4+ 6)
    const uint32_t sp_max = (uint32_t)s->cfgs[0].charge_max + 2u;
    launch_pack_keys(sp, iz, ir, pz, pr, n, RI.nz, RI.nr, RI.cell_base, rs.id_next, sp_max, s->A.key + o,
                     s->A.id + o, dbad, grid_for(s, 8), s->stream);
    CK(cudaGetLastError());
    const float* src[5] = {pz, pr, vz, vr, vt};
    float* dst[5] = {s->A.pz + o, s->A.pr + o, s->A.vz + o, s->A.vr + o, s->A.vt + o};
    for (int k = 0; k < 5; ++k)   // (a host load has already put them in place)
        if (src[k] != dst[k]) CK(cudaMemcpyAsync(dst[k], src[k], n * 4, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(&bad, dbad, 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (bad) return fail(s, PD_ERR_ARG, "a device particle is out of range");
    d.n_slots += (uint64_t)n;
    rs.id_next += (uint32_t)n;
    CK(cudaMemcpyAsync(&s->st->n_slots, &d.n_slots, 8, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(&s->rs[run].id_next, &rs.id_next, 4, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->primed = false;
    return PD_OK;
}

pd_status run_scalars(pd_sim* s, int run, pd_scalars* out) {
    if (!s || !out || run < 0 || run >= s->R) return PD_ERR_ARG;
    if (s->spc_version != s->version) {
        // one pass counts every run (an ensemble's runs are read one after another)
        s->spc_host.assign((size_t)s->R * NSP, 0ull);
        CK(cudaMemsetAsync(s->spc, 0, (size_t)s->R * NSP * 8, s->stream));
        launch_species_count_all(s->A, s->st, kparams(s, 1), s->spc, grid_for(s, 4), s->stream);
        CK(cudaMemcpyAsync(s->spc_host.data(), s->spc, (size_t)s->R * NSP * 8, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        s->spc_version = s->version;
    }
    unsigned long long cnt[NSP];
    for (int k = 0; k < NSP; ++k) cnt[k] = s->spc_host[(size_t)run * NSP + k];
    RunState d;
    pd_status r = read_run(s, run, &d);
    if (r != PD_OK) return r;
    std::memset(out, 0, sizeof(*out));
    const pd_config& c = s->cfgs[run];
    out->t = (double)s->step * c.dt;
    out->V = d.V;
    out->I_gap = d.I_gap;
    // Eq. (21) over the heavy species: ionization degree and mean ion charge
    double ions = 0.0, qsum = 0.0;
    for (int sp = SP_CUP; sp < NSP; ++sp) {
        ions += (double)cnt[sp];
        qsum += (double)ZQ[sp] * (double)cnt[sp];
    }
    const double all = (double)cnt[SP_CU] + ions;
    out->gamma = all > 0 ? ions / all : 0.0;
    out->Qbar = ions > 0 ? qsum / ions : 0.0;
    double heavy_back = 0;
    for (int sp = 1; sp < NSP; ++sp) heavy_back += (double)d.ctr[C_ABS + 0 * NSP + sp];
    // net Cu leaving the cathode: injected and sputtered neutrals less the heavies it absorbed
    out->mass = M_CU * c.weight * ((double)d.ctr[C_EMIT_CU] + (double)d.ctr[C_SPUT_C] - heavy_back);
    out->charge = d.charge_cathode;
    out->erosion = out->charge != 0 ? out->mass / out->charge : 0.0;
    out->sgmax[0] = s->cc.sgmax[0];
    out->sgmax[1] = s->cc.sgmax[1];
    out->poisson_relres = d.relres;
    out->poisson_cycles = d.cycles;
    out->poisson_relres_max = d.relres_max;
    out->poisson_relres0 = d.relres0;
    for (int k = 0; k < 3; ++k) out->absorbed_energy[k] = d.absorbed_energy[k];
    int64_t tot = 0;
    for (int sp = 0; sp < NSP; ++sp) {
        out->count[sp] = (int64_t)cnt[sp];
        tot += (int64_t)cnt[sp];
    }
    out->n_particles = tot;
    out->step = s->step;
    return PD_OK;
}

pd_status run_density(pd_sim* s, int run, int species, double* out) {
    if (!s || !out || species < 0 || species >= NSP || run < 0 || run >= s->R) return PD_ERR_ARG;
    const pd_config& c = s->cfgs[run];
    const RunInfo& RI = s->runs[run];
    const size_t nodes = total_nodes(s);
    CK(cudaMemsetAsync(s->diag, 0, nodes * 8, s->stream));
    launch_density(s->A, s->st, kparams(s, 1), run, species, s->diag, grid_for(s, 8), s->stream);
    const size_t rn = run_nodes(c);
    std::vector<long long> h(rn);
    CK(cudaMemcpyAsync(h.data(), s->diag + RI.node_base, rn * 8, cudaMemcpyDeviceToHost, s->stream));
    DevState d;
    pd_status r = sync_check(s, &d);
    if (r != PD_OK) return r;
    for (int i = 0; i < RI.nzn; ++i)
        for (int j = 0; j < RI.nrn; ++j) {
            const size_t k = (size_t)i * RI.nrn + j;
            out[k] = c.weight * (double)h[k] / 4294967296.0 / node_volume(c, i, j);
        }
    return PD_OK;
}

pd_status run_spectrum(pd_sim* s, int run, int species, double lo, double hi, int nbins, uint64_t* out) {
    if (!s || !out || species < 0 || species >= NSP || nbins < 1 || nbins > 4096 || !(hi > lo) || run < 0 ||
        run >= s->R)
        return PD_ERR_ARG;
    CK(cudaMemsetAsync(s->hist, 0, (size_t)nbins * 8, s->stream));
    launch_spectrum(s->A, s->st, kparams(s, 1), run, species, lo, hi, nbins, s->hist, grid_for(s, 8), s->stream);
    CK(cudaMemcpyAsync(out, s->hist, (size_t)nbins * 8, cudaMemcpyDeviceToHost, s->stream));
    DevState d;
    return sync_check(s, &d);
}

}  // namespace

extern "C" {

pd_status pd_config_default(pd_config* c) {
    if (!c) return PD_ERR_ARG;
    std::memset(c, 0, sizeof(*c));
    c->struct_size = sizeof(pd_config);
    c->version = PD_CONFIG_VERSION;
    c->geometry = PD_GEOM_RZ;
    c->nz = 64;
    c->nr = 64;
    c->dz = 6e-6 / 64;
    c->dr = 6e-6 / 64;
    c->depth = 1.0;
    c->dt = 1e-15;
    c->heavy_subcycle = 10;
    c->weight = 100.0;
    c->seed = 1;
    c->run = 0;
    c->field_mode = PD_FIELD_POISSON;
    c->inject_on = 1;
    c->di_on = 1;
    c->di_split_mode = 0;
    c->coll_dt_scale = 1.0;
    c->V0 = 2.9e3;
    c->R_ohm = 1e3;
    c->C_farad = 1e-12;
    c->beta = 35.0;
    c->tip_radius = 100e-9;
    c->work_function = 4.5;
    c->neutral_ratio = 0.03;
    c->neutral_T = 2000.0;
    c->poisson_tol = 1e-8;
    c->poisson_max_cycles = 60;
    c->heavy_coll = 0;
    c->charge_max = 2;
    c->coulomb = 0;
    c->coulomb_lnl = 10.0;
    c->sputter = 0;
    c->reserved1 = 0;
    c->sputter_T = 23209.0;
    c->capacity = 1 << 16;
    return PD_OK;
}

pd_status pd_ensemble_workspace_size(const pd_config* cfgs, int n, size_t* bytes) {
    std::string msg;
    pd_status r = validate(cfgs, n, msg);
    if (r != PD_OK) return r;
    if (!bytes) return PD_ERR_ARG;
    *bytes = make_layout(std::vector<pd_config>(cfgs, cfgs + n)).total;
    return PD_OK;
}

pd_status pd_workspace_size(const pd_config* c, size_t* bytes) { return pd_ensemble_workspace_size(c, 1, bytes); }

pd_status pd_ensemble_create(const pd_config* cfgs, int n, void* ws, size_t bytes, void* stream, pd_ensemble** out) {
    return create_common(cfgs, n, ws, bytes, stream, out);
}

pd_status pd_create(const pd_config* c, void* ws, size_t bytes, void* stream, pd_sim** out) {
    return create_common(c, 1, ws, bytes, stream, out);
}

pd_status pd_run_count(pd_sim* s, int* n) {
    if (!s || !n) return PD_ERR_ARG;
    *n = s->R;
    return PD_OK;
}

pd_status pd_run_layout(pd_sim* s, int run, int64_t* cell_base, int64_t* node_base) {
    if (!s || run < 0 || run >= s->R) return PD_ERR_ARG;
    if (cell_base) *cell_base = s->runs[run].cell_base;
    if (node_base) *node_base = s->runs[run].node_base;
    return PD_OK;
}

pd_status pd_set_cross_section(pd_sim* s, int ch, const double* E, const double* sig, int n, double threshold) {
    if (!s) return PD_ERR_ARG;
    if (ch < 0 || ch >= NCH || n < 2 || !E || !sig) return fail(s, PD_ERR_ARG, "bad cross-section arguments");
    for (int a = 0; a + 1 < n; ++a)
        if (!(E[a + 1] > E[a])) return fail(s, PD_ERR_ARG, "cross-section energies must ascend");
    for (int k = 0; k < XS_N; ++k) {
        const double e = (double)s->h_xsE[k];
        double v;
        if (e <= E[0]) v = sig[0];
        else if (e >= E[n - 1]) v = sig[n - 1];
        else {
            int a = 0;
            while (E[a + 1] <= e) ++a;
            const double t = (e - E[a]) / (E[a + 1] - E[a]);
            v = sig[a] + t * (sig[a + 1] - sig[a]);
        }
        if (e < threshold) v = 0.0;
        if (ch == CH_DI && !s->cfgs[0].di_on) v = 0.0;
        s->h_xs[ch][k] = (float)v;
    }
    s->eth[ch] = threshold;
    update_collision_consts(s);
    drop_graph(s);
    CK(cudaMemcpyAsync(s->xs + (size_t)ch * XS_N, s->h_xs[ch], XS_N * 4, cudaMemcpyHostToDevice, s->stream));
    return upload_ck(s);
}

pd_status pd_set_sputter_yield(pd_sim* s, const double* E, const double* Y, int n) {
    if (!s) return PD_ERR_ARG;
    if (n < 2 || !E || !Y) return fail(s, PD_ERR_ARG, "bad sputtering-yield arguments");
    for (int a = 0; a + 1 < n; ++a)
        if (!(E[a + 1] > E[a])) return fail(s, PD_ERR_ARG, "yield energies must ascend");
    for (int k = 0; k < XS_N; ++k) {
        const double e = (double)s->h_xsE[k];
        double v;
        if (e <= E[0]) v = Y[0];
        else if (e >= E[n - 1]) v = Y[n - 1];
        else {
            int a = 0;
            while (E[a + 1] <= e) ++a;
            const double t = (e - E[a]) / (E[a + 1] - E[a]);
            v = Y[a] + t * (Y[a + 1] - Y[a]);
        }
        s->h_ytab[k] = (float)v;
    }
    drop_graph(s);
    CK(cudaMemcpyAsync(s->ytab, s->h_ytab, sizeof(s->h_ytab), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return PD_OK;
}

pd_status pd_load_particles(pd_sim* s, int64_t n, const uint8_t* sp, const int32_t* iz, const int32_t* ir,
                            const float* pz, const float* pr, const float* vz, const float* vr, const float* vt) {
    return load_host(s, 0, n, sp, iz, ir, pz, pr, vz, vr, vt);
}

pd_status pd_load_particles_run(pd_sim* s, int run, int64_t n, const uint8_t* sp, const int32_t* iz,
                                const int32_t* ir, const float* pz, const float* pr, const float* vz, const float* vr,
                                const float* vt) {
    return load_host(s, run, n, sp, iz, ir, pz, pr, vz, vr, vt);
}

pd_status pd_load_particles_device(pd_sim* s, int64_t n, const uint8_t* sp, const int32_t* iz, const int32_t* ir,
                                   const float* pz, const float* pr, const float* vz, const float* vr,
                                   const float* vt) {
    return load_device(s, 0, n, sp, iz, ir, pz, pr, vz, vr, vt);
}

pd_status pd_load_particles_device_run(pd_sim* s, int run, int64_t n, const uint8_t* sp, const int32_t* iz,
                                       const int32_t* ir, const float* pz, const float* pr, const float* vz,
                                       const float* vr, const float* vt) {
    return load_device(s, run, n, sp, iz, ir, pz, pr, vz, vr, vt);
}

pd_status pd_set_field(pd_sim* s, const double* Ez, const double* Er) {
    if (!s || !Ez || !Er) return PD_ERR_ARG;
    const size_t nodes = total_nodes(s);
    std::vector<float2> h(nodes);
    for (size_t k = 0; k < nodes; ++k) h[k] = make_float2((float)Ez[k], (float)Er[k]);
    CK(cudaMemcpyAsync(s->E, h.data(), nodes * 8, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return PD_OK;
}

pd_status pd_inject_cathode(pd_sim* s, int enable) {
    if (!s) return PD_ERR_ARG;
    if (enable && s->cfgs[0].geometry != PD_GEOM_RZ) return fail(s, PD_ERR_ARG, "injection needs r-z");
    for (int r = 0; r < s->R; ++r) {
        pd_config c = s->cfgs[r];
        c.inject_on = enable ? 1 : 0;
        s->ic[r] = make_injection(c);
    }
    s->any_inject = false;
    for (int r = 0; r < s->R; ++r) s->any_inject = s->any_inject || s->ic[r].ntip > 0;
    drop_graph(s);
    CK(cudaMemcpyAsync(s->ic_dev, s->ic.data(), s->R * sizeof(InjectConsts), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return PD_OK;
}

pd_status pd_set_graph_mode(pd_sim* s, int enable, int poisson_cycles) {
    if (!s || poisson_cycles < 0) return PD_ERR_ARG;
    drop_graph(s);
    s->graph_on = enable != 0;
    s->graph_cycles = poisson_cycles > 0 ? poisson_cycles : 4;
    return PD_OK;
}

pd_status pd_step(pd_sim* s, int64_t n_steps) {
    if (!s) return PD_ERR_ARG;
    ++s->version;
    if (n_steps < 0) return fail(s, PD_ERR_ARG, "n_steps < 0");
    // RunState::relres_max of every run restarts with this call
    CK(cudaMemset2DAsync(&s->rs[0].relres_max, sizeof(RunState), 0, sizeof(double), (size_t)s->R, s->stream));
    if (!s->primed) {
        drop_graph(s);
        pd_status r = prime(s);
        if (r != PD_OK) return r;
    }
    int64_t left = n_steps;
    while (left > 0) {
        const int G = graph_period(s);
        if (s->graph_on && s->sorted_valid && s->step % G == 0 && left >= G) {
            if (!s->gexec) {
                pd_status r = build_graph(s);
                if (r != PD_OK) return r;
            }
            CK(cudaGraphLaunch(s->gexec, s->stream));
            for (int k = 0; k < PD_NKERNELS; ++k) s->launches[k] += s->graph_launches[k];
            s->step += G;
            left -= G;
            continue;
        }
        pd_status r = issue_step(s, false);
        if (r != PD_OK) return r;
        --left;
    }
    CK(cudaGetLastError());
    return PD_OK;
}

pd_status pd_ensemble_step(pd_ensemble* s, int64_t n_steps) { return pd_step(s, n_steps); }

pd_status pd_synchronize(pd_sim* s) {
    if (!s) return PD_ERR_ARG;
    DevState d;
    return sync_check(s, &d);
}

pd_status pd_get_scalars(pd_sim* s, pd_scalars* out) { return run_scalars(s, 0, out); }
pd_status pd_ensemble_get_scalars(pd_ensemble* s, int run, pd_scalars* out) { return run_scalars(s, run, out); }

pd_status pd_get_run_counters(pd_sim* s, int run, uint64_t* out) {
    if (!s || !out || run < 0 || run >= s->R) return PD_ERR_ARG;
    RunState d;
    pd_status r = read_run(s, run, &d);
    if (r != PD_OK) return r;
    for (int k = 0; k < NCOUNTERS; ++k) out[k] = d.ctr[k];
    return PD_OK;
}

pd_status pd_get_counters(pd_sim* s, uint64_t* out) { return pd_get_run_counters(s, 0, out); }

pd_status pd_particle_slots(pd_sim* s, int64_t* slots) {
    if (!s || !slots) return PD_ERR_ARG;
    DevState d;
    pd_status r = sync_check(s, &d);
    if (r != PD_OK) return r;
    *slots = (int64_t)d.n_slots;
    return PD_OK;
}

pd_status pd_get_sort_stats(pd_sim* s, pd_sort_stats* out) {
    if (!s || !out) return PD_ERR_ARG;
    DevState d;
    CK(cudaMemcpyAsync(&d, s->st, sizeof(d), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    // (read without the error check, so that it also reports a failed sort)
    out->faults = d.sort_fault;
    out->relayouts = d.n_relayout;
    out->bin_slots = d.tail_base;   // heavy bins with their slack, then the electron bins
    out->live = d.n_live + d.n_e;
    out->steps_since = d.since;
    return PD_OK;
}

pd_status pd_get_bins(pd_sim* s, uint32_t* start, uint32_t* count, int64_t* nbins) {
    if (!s || !nbins) return PD_ERR_ARG;
    const size_t nb = (size_t)s->L.ncell * (size_t)s->L.nsp;
    *nbins = (int64_t)nb;
    if (!start && !count) return PD_OK;
    if (!start || !count) return PD_ERR_ARG;
    DevState d;
    pd_status r = sync_check(s, &d);
    if (r != PD_OK) return r;
    CK(cudaMemcpyAsync(start, s->off, (nb + 1) * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(count, s->bcnt, nb * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return PD_OK;
}

pd_status pd_get_particles(pd_sim* s, uint32_t* id, int32_t* run, uint8_t* sp, int32_t* iz, int32_t* ir, float* pz,
                           float* pr, float* vz, float* vr, float* vt) {
    if (!s) return PD_ERR_ARG;
    DevState d;
    pd_status r = sync_check(s, &d);
    if (r != PD_OK) return r;
    const size_t n = d.n_slots;
    if (n == 0) return PD_OK;
    std::vector<uint32_t> key(n);
    std::vector<uint16_t> cell_run;
    CK(cudaMemcpyAsync(key.data(), s->A.key, n * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(id, s->A.id, n * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(pz, s->A.pz, n * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(pr, s->A.pr, n * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(vz, s->A.vz, n * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(vr, s->A.vr, n * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(vt, s->A.vt, n * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (size_t q = 0; q < n; ++q) {
        if (key[q] == DEAD) {
            sp[q] = 255;
            iz[q] = -1;
            ir[q] = -1;
            if (run) run[q] = -1;
            continue;
        }
        const uint32_t g = key[q] & 0xFFFFFFu;
        const int rr = s->h_cell_run[g];
        const RunInfo& RI = s->runs[rr];
        const uint32_t lc = g - RI.cell_base;
        sp[q] = (uint8_t)((key[q] >> 24) & 7u);
        iz[q] = (int32_t)(lc / (uint32_t)RI.nr);
        ir[q] = (int32_t)(lc % (uint32_t)RI.nr);
        if (run) run[q] = rr;
    }
    return PD_OK;
}

pd_status pd_get_rho(pd_sim* s, int64_t* rho_e, int64_t* rho_h) {
    if (!s) return PD_ERR_ARG;
    const size_t nodes = total_nodes(s);
    if (rho_e) CK(cudaMemcpyAsync(rho_e, s->rho_e, nodes * 8, cudaMemcpyDeviceToHost, s->stream));
    if (rho_h) CK(cudaMemcpyAsync(rho_h, s->rho_h, nodes * 8, cudaMemcpyDeviceToHost, s->stream));
    DevState d;
    return sync_check(s, &d);
}

pd_status pd_get_phi(pd_sim* s, double* phi) {
    if (!s || !phi) return PD_ERR_ARG;
    CK(cudaMemcpyAsync(phi, s->phi, total_nodes(s) * 8, cudaMemcpyDeviceToHost, s->stream));
    DevState d;
    return sync_check(s, &d);
}

pd_status pd_get_rho_phi(pd_sim* s, double* rho, double* phi) {
    if (!s || !rho || !phi) return PD_ERR_ARG;
    const size_t nodes = total_nodes(s);
    std::vector<long long> he(nodes), hh(nodes);
    CK(cudaMemcpyAsync(he.data(), s->rho_e, nodes * 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(hh.data(), s->rho_h, nodes * 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(phi, s->phi, nodes * 8, cudaMemcpyDeviceToHost, s->stream));
    DevState d;
    pd_status r = sync_check(s, &d);
    if (r != PD_OK) return r;
    for (int run = 0; run < s->R; ++run) {
        const pd_config& c = s->cfgs[run];
        const RunInfo& RI = s->runs[run];
        for (int i = 0; i < RI.nzn; ++i)
            for (int j = 0; j < RI.nrn; ++j) {
                const size_t k = RI.node_base + (size_t)i * RI.nrn + j;
                rho[k] = QE * c.weight * (double)(he[k] + hh[k]) / 4294967296.0 / node_volume(c, i, j);
            }
    }
    return PD_OK;
}

pd_status pd_warmstart_pairs(pd_sim* s, int kind, float* x, float* t) {
    if (!s || !x || !t || (kind != PD_PAIRS_ABSOLUTE && kind != PD_PAIRS_DELTA && kind != PD_PAIRS_EXTRAP))
        return PD_ERR_ARG;
    if (s->cfgs[0].field_mode != PD_FIELD_POISSON) return fail(s, PD_ERR_STATE, "warm start needs the Poisson field");
    if (!s->primed) {
        pd_status r = prime(s);
        if (r != PD_OK) return r;
    }
    if (s->solves < 1 + kind)
        return fail(s, PD_ERR_STATE, "not enough solves since create or load for these pairs");
    const int form = kind == PD_PAIRS_DELTA ? WARM_DELTA : kind == PD_PAIRS_EXTRAP ? WARM_EXTRAP : WARM_ABSOLUTE;
    warm_inputs(s->field, s->whist, form, s->runs_dev, s->rmax, x, s->stream);
    warm_targets(s->field, s->phi, s->whist, form, s->runs_dev, s->rmax, t, s->stream);
    CK(cudaGetLastError());
    return PD_OK;
}

pd_status pd_set_warm_start(pd_sim* s, int mode, pd_net* net) {
    if (!s) return PD_ERR_ARG;
    if (mode != PD_WARM_PREVIOUS && mode != PD_WARM_COLD && mode != PD_WARM_LEARNED && mode != PD_WARM_LEARNED_DELTA &&
        mode != PD_WARM_EXTRAPOLATE && mode != PD_WARM_LEARNED_EXTRAP)
        return fail(s, PD_ERR_ARG, "bad warm-start mode");
    if (mode != PD_WARM_PREVIOUS && s->cfgs[0].field_mode != PD_FIELD_POISSON)
        return fail(s, PD_ERR_STATE, "warm start needs the Poisson field");
    const bool learned = mode == PD_WARM_LEARNED || mode == PD_WARM_LEARNED_DELTA || mode == PD_WARM_LEARNED_EXTRAP;
    if (learned) {
        if (!net) return fail(s, PD_ERR_ARG, "learned warm start needs a network");
        if (net_max_nodes(net) < (int64_t)total_nodes(s))
            return fail(s, PD_ERR_ARG, "network holds fewer nodes than the simulation");
        // batches of runs of one grid shape
        std::vector<pd_sim::Group> groups;
        std::vector<uint32_t> bases;
        std::vector<int> done(s->R, 0);
        for (int r = 0; r < s->R; ++r) {
            if (done[r]) continue;
            pd_sim::Group g{0, s->cfgs[r].nz + 1, s->cfgs[r].nr + 1, (int)bases.size()};
            for (int q = r; q < s->R; ++q)
                if (!done[q] && s->cfgs[q].nz == s->cfgs[r].nz && s->cfgs[q].nr == s->cfgs[r].nr) {
                    bases.push_back(s->node_base[q]);
                    done[q] = 1;
                    ++g.B;
                }
            groups.push_back(g);
        }
        CK(cudaMemcpyAsync(s->grp_base, bases.data(), bases.size() * 4, cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        s->groups = groups;
    }
    drop_graph(s);
    s->warm_mode = mode;
    s->warm_net = learned ? net : nullptr;
    return PD_OK;
}

pd_status pd_save(pd_sim* s, const char* path) {
    if (!s || !path) return PD_ERR_ARG;
    DevState d;
    pd_status r = sync_check(s, &d);
    if (r != PD_OK) return r;
    File F(std::fopen(path, "wb"));
    if (!F.f) return fail(s, PD_ERR_ARG, std::string("cannot open ") + path);
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, CKPT_MAGIC, 8);
    h.version = CKPT_VERSION;
    h.nruns = (uint32_t)s->R;
    h.cfg_size = sizeof(pd_config);
    h.runstate_size = sizeof(RunState);
    h.devstate_size = sizeof(DevState);
    h.sorted_valid = s->sorted_valid ? 1u : 0u;
    h.primed = s->primed ? 1u : 0u;
    h.step = s->step;
    h.n_slots = d.n_slots;
    h.n_off = (uint64_t)s->L.nbins_pad + 1;
    h.nodes = total_nodes(s);
    h.cap = s->L.cap;
    bool ok = F.put(&h, sizeof(h)) && F.put(s->cfgs.data(), s->cfgs.size() * sizeof(pd_config)) &&
              F.put(s->h_xs, sizeof(s->h_xs)) && F.put(s->eth, sizeof(s->eth)) &&
              F.put(s->h_ytab, sizeof(s->h_ytab)) && F.put(&d, sizeof(d));
    if (!ok) return fail(s, PD_ERR_ARG, "checkpoint write failed");
    const size_t nodes = (size_t)h.nodes, n = (size_t)h.n_slots;
    const void* arrays[7] = {s->A.key, s->A.pz, s->A.pr, s->A.vz, s->A.vr, s->A.vt, s->A.id};
    if ((r = dev_to_file(s, F, s->rs, (size_t)s->R * sizeof(RunState))) != PD_OK) return r;
    if ((r = dev_to_file(s, F, s->off, (size_t)h.n_off * 4)) != PD_OK) return r;
    if ((r = dev_to_file(s, F, s->bcnt, (size_t)(h.n_off - 1) * 4)) != PD_OK) return r;
    if ((r = dev_to_file(s, F, s->rho_e, nodes * 8)) != PD_OK) return r;
    if ((r = dev_to_file(s, F, s->rho_h, nodes * 8)) != PD_OK) return r;
    if ((r = dev_to_file(s, F, s->E, nodes * 8)) != PD_OK) return r;
    if ((r = dev_to_file(s, F, s->phi, nodes * 8)) != PD_OK) return r;
    for (int a = 0; a < 7; ++a)
        if ((r = dev_to_file(s, F, arrays[a], n * 4)) != PD_OK) return r;
    if (std::fflush(F.f) != 0) return fail(s, PD_ERR_ARG, "checkpoint write failed");
    return PD_OK;
}

pd_status pd_load(pd_sim* s, const char* path) {
    if (!s || !path) return PD_ERR_ARG;
    ++s->version;
    DevState cur;
    pd_status r = sync_check(s, &cur);
    if (r != PD_OK) return r;
    File F(std::fopen(path, "rb"));
    if (!F.f) return fail(s, PD_ERR_ARG, std::string("cannot open ") + path);
    CkptHeader h;
    if (!F.get(&h, sizeof(h)) || std::memcmp(h.magic, CKPT_MAGIC, 8) != 0 || h.version != CKPT_VERSION)
        return fail(s, PD_ERR_ARG, "not a checkpoint of this library version");
    if (h.nruns != (uint32_t)s->R || h.cfg_size != sizeof(pd_config) || h.runstate_size != sizeof(RunState) ||
        h.devstate_size != sizeof(DevState) || h.n_off != (uint64_t)s->L.nbins_pad + 1 ||
        h.nodes != total_nodes(s) || h.cap != s->L.cap)
        return fail(s, PD_ERR_ARG, "checkpoint was written by a simulation of another shape");
    if (h.n_slots > s->L.cap) return fail(s, PD_ERR_CAPACITY, "checkpoint holds more slots than the capacity");
    std::vector<pd_config> cf(s->R);
    if (!F.get(cf.data(), cf.size() * sizeof(pd_config))) return fail(s, PD_ERR_ARG, "checkpoint file is truncated");
    for (int k = 0; k < s->R; ++k)
        if (!same_config(cf[k], s->cfgs[k])) return fail(s, PD_ERR_ARG, "checkpoint configs differ from this simulation's");
    float xs[NCH][XS_N];
    double eth[NCH];
    float ytab[XS_N];
    DevState d;
    if (!F.get(xs, sizeof(xs)) || !F.get(eth, sizeof(eth)) || !F.get(ytab, sizeof(ytab)) || !F.get(&d, sizeof(d)))
        return fail(s, PD_ERR_ARG, "checkpoint file is truncated");
    if (d.n_slots != h.n_slots) return fail(s, PD_ERR_ARG, "inconsistent checkpoint");
    drop_graph(s);
    const size_t nodes = (size_t)h.nodes, n = (size_t)h.n_slots;
    void* arrays[7] = {s->A.key, s->A.pz, s->A.pr, s->A.vz, s->A.vr, s->A.vt, s->A.id};
    if ((r = file_to_dev(s, F, s->rs, (size_t)s->R * sizeof(RunState))) != PD_OK) return r;
    if ((r = file_to_dev(s, F, s->off, (size_t)h.n_off * 4)) != PD_OK) return r;
    if ((r = file_to_dev(s, F, s->bcnt, (size_t)(h.n_off - 1) * 4)) != PD_OK) return r;
    if ((r = file_to_dev(s, F, s->rho_e, nodes * 8)) != PD_OK) return r;
    if ((r = file_to_dev(s, F, s->rho_h, nodes * 8)) != PD_OK) return r;
    if ((r = file_to_dev(s, F, s->E, nodes * 8)) != PD_OK) return r;
    if ((r = file_to_dev(s, F, s->phi, nodes * 8)) != PD_OK) return r;
    for (int a = 0; a < 7; ++a)
        if ((r = file_to_dev(s, F, arrays[a], n * 4)) != PD_OK) return r;
    // slots past the saved ones are free; a checkpoint is taken between
    // steps, when no bin has traffic, no mover is pending and no slot is a hole
    CK(cudaMemsetAsync(s->A.key + n, 0xFF, (size_t)(s->L.cap - n) * 4, s->stream));
    const size_t nbp = (size_t)s->L.nbins_pad;
    CK(cudaMemsetAsync(s->count, 0, nbp * 4, s->stream));
    CK(cudaMemsetAsync(s->outc, 0, nbp * 4, s->stream));
    CK(cudaMemsetAsync(s->act, 0, nbp * 4, s->stream));
    CK(cudaMemsetAsync(s->net, 0, nbp * 4, s->stream));
    CK(cudaMemsetAsync(s->mm, 0, (size_t)s->L.words_pad * 4, s->stream));
    std::memcpy(s->h_xs, xs, sizeof(xs));
    std::memcpy(s->eth, eth, sizeof(eth));
    std::memcpy(s->h_ytab, ytab, sizeof(ytab));
    update_collision_consts(s);
    CK(cudaMemcpyAsync(s->xs, s->h_xs, sizeof(s->h_xs), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->ytab, s->h_ytab, sizeof(s->h_ytab), cudaMemcpyHostToDevice, s->stream));
    d.error = 0;
    d.load_bad = 0;
    CK(cudaMemcpyAsync(s->st, &d, sizeof(d), cudaMemcpyHostToDevice, s->stream));
    r = upload_ck(s);
    if (r != PD_OK) return r;
    s->step = h.step;
    s->solves = 0;            // the warm-start history is not part of the checkpoint
    s->sorted_valid = h.sorted_valid != 0;
    s->primed = h.primed != 0;
    CK(cudaStreamSynchronize(s->stream));
    return PD_OK;
}

pd_status pd_get_field(pd_sim* s, double* Ez, double* Er) {
    if (!s || !Ez || !Er) return PD_ERR_ARG;
    const size_t nodes = total_nodes(s);
    std::vector<float2> h(nodes);
    CK(cudaMemcpyAsync(h.data(), s->E, nodes * 8, cudaMemcpyDeviceToHost, s->stream));
    DevState d;
    pd_status r = sync_check(s, &d);
    if (r != PD_OK) return r;
    for (size_t k = 0; k < nodes; ++k) {
        Ez[k] = h[k].x;
        Er[k] = h[k].y;
    }
    return PD_OK;
}

pd_status pd_get_density_map(pd_sim* s, int species, double* out) { return run_density(s, 0, species, out); }
pd_status pd_get_run_density_map(pd_sim* s, int run, int species, double* out) {
    return run_density(s, run, species, out);
}

pd_status pd_get_energy_spectrum(pd_sim* s, int species, double lo, double hi, int nbins, uint64_t* out) {
    return run_spectrum(s, 0, species, lo, hi, nbins, out);
}
pd_status pd_get_run_energy_spectrum(pd_sim* s, int run, int species, double lo, double hi, int nbins,
                                     uint64_t* out) {
    return run_spectrum(s, run, species, lo, hi, nbins, out);
}

pd_status pd_profile_enable(pd_sim* s, int enable) {
    if (!s) return PD_ERR_ARG;
    s->prof = enable != 0;
    if (s->prof) fill_event_pool(s);
    return PD_OK;
}

pd_status pd_profile_read(pd_sim* s, double* ms, uint64_t* launches) {
    if (!s) return PD_ERR_ARG;
    for (int k = 0; k < PD_NKERNELS; ++k) {
        if (launches) launches[k] = s->launches[k];
        s->launches[k] = 0;
    }
    return collect_profile(s, ms);
}

pd_status pd_get_tuning(pd_sim* s, pd_tuning* out) {
    if (!s || !out) return PD_ERR_ARG;
    *out = s->tune;
    return PD_OK;
}

pd_status pd_set_tuning(pd_sim* s, const pd_tuning* t) {
    if (!s || !t) return PD_ERR_ARG;
    if (!tuning_ok(*t)) return fail(s, PD_ERR_ARG, "launch shape out of range");
    drop_graph(s);
    apply_tuning(s, *t);
    return PD_OK;
}

pd_status pd_autotune(pd_sim* s, int steps_per_trial, pd_tuning* out) {
    if (!s) return PD_ERR_ARG;
    ++s->version;
    if (steps_per_trial < 1 || steps_per_trial > 64) return fail(s, PD_ERR_ARG, "steps_per_trial must be in 1..64");
    if (!s->primed) {
        pd_status r = prime(s);
        if (r != PD_OK) return r;
    }
    drop_graph(s);
    const bool prof0 = s->prof;
    fill_event_pool(s);
    pd_status r = collect_profile(s, nullptr);      // earlier records are discarded
    uint64_t launches0[PD_NKERNELS];
    std::memcpy(launches0, s->launches, sizeof(launches0));
    struct Knob {
        int* v;
        int kernel;
        std::vector<int> cand;
    };
    pd_tuning t = s->tune;
    std::vector<Knob> knobs = {
        {&t.push_blocks_per_sm, K_PUSH, {3, 4, 6, 8, 12, 16}},
        {&t.bincount_blocks_per_sm, K_SCAN_BINS, {2, 4, 8, 16}},
        {&t.scatter_blocks_per_sm, K_SCATTER, {2, 3, 4, 6, 8, 12, 16}},
        {&t.ncand_blocks_per_sm, K_NCAND, {2, 4, 8, 16}},
        {&t.collide_blocks_per_sm, K_COLLIDE, {4, 8, 16, 32}},
    };
    if (s->cfgs[0].field_mode == PD_FIELD_POISSON) {
        knobs.push_back({&t.mg_threads, K_POISSON, {64, 128, 256, 512}});
        knobs.push_back({&t.mg_max_blocks, K_POISSON, {76, 152, 304, 608, 1216}});
    }
    // time the knob's kernel for one value: an untimed step, then
    // steps_per_trial profiled ones
    auto trial = [&](int kid, double* ms) -> pd_status {
        apply_tuning(s, t);
        s->prof = false;
        pd_status q = issue_step(s, false);
        s->prof = true;
        for (int k = 0; k < steps_per_trial && q == PD_OK; ++k) q = issue_step(s, false);
        s->prof = false;
        double acc[PD_NKERNELS];
        const pd_status c = collect_profile(s, acc);
        if (q != PD_OK) return q;
        if (c != PD_OK) return c;
        DevState d;
        q = sync_check(s, &d);
        *ms = acc[kid];
        return q;
    };
    for (size_t kn = 0; kn < knobs.size() && r == PD_OK; ++kn) {
        Knob& K = knobs[kn];
        // the current value first: another must beat it by 2 % to replace it
        std::vector<int> order = {*K.v};
        for (int v : K.cand)
            if (v != *K.v) order.push_back(v);
        int best = *K.v;
        double best_ms = 0.0;
        for (size_t q = 0; q < order.size() && r == PD_OK; ++q) {
            *K.v = order[q];
            double ms = 0.0;
            r = trial(K.kernel, &ms);
            if (r == PD_OK && (q == 0 || ms < 0.98 * best_ms)) {
                best = order[q];
                best_ms = ms;
            }
        }
        *K.v = best;
    }
    apply_tuning(s, t);
    std::memcpy(s->launches, launches0, sizeof(launches0));
    s->prof = prof0;
    if (out) *out = s->tune;
    return r;
}

const char* pd_kernel_name(int k) { return (k >= 0 && k < PD_NKERNELS) ? KNAMES[k] : "?"; }

const char* pd_last_error(const pd_sim* s) { return s ? s->err.c_str() : "null simulation"; }

void pd_destroy(pd_sim* s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    drop_graph(s);
    if (s->capture_stream) cudaStreamDestroy(s->capture_stream);
    for (auto& r : s->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : s->pool) cudaEventDestroy(e);
    field_free(s->field);
    delete s;
}

}  // extern "C"
