// pd_field.h -- Poisson solve (Eq. (8)) and E = -grad(phi) on the r-z node
// grids of all runs of a simulation, batched.
#pragma once
#include <cstddef>
#include <vector>

#include "pd.h"
#include "pd_internal.cuh"

namespace pd {

constexpr int MG_MAX_LEVELS = 12;
constexpr int MG_DIRECT_MAX = 256;      // coarsest levels up to this many unknowns are solved by their inverse

// one level of one run's correction multigrid (float)
struct MGLevel {
    int nz, nr;              // cells
    float *e, *e2, *f;       // correction (post-smoothed), pre-smoothed correction, right-hand side (nodes)
    float *ap, *am, *b;      // per radial node j: radial face and axial coefficients
    float* dinv;             // 1 / (ap + am + 2 b)
};

// the double-precision problem of one run (level 0)
struct MGTop {
    int nz, nr;
    double* phi;             // the run's potential (the simulation's phi at the run's node base)
    double* bf;              // right-hand side b of the discrete Eq. (8) (nodes)
    double *ap, *am, *b;     // coefficients per radial node
    double* dg;              // diagonal ap + am + 2 b per radial node
    double* cr;              // b = (rho_e + rho_h) cr[j] on interior rows (plus the anode row's b V)
    double* iv;              // 1 / Verboncoeur volume of an interior node at j
    double idz, i2dz, i2dr;  // 1 / dz, 1 / (2 dz), 1 / (2 dr)
};

struct FieldSolver {
    int nruns = 0;
    int max_levels = 0;                 // deepest hierarchy over the runs
    std::vector<int> nlev;              // levels of each run
    std::vector<MGLevel> host_lev;      // [run * MG_MAX_LEVELS + l]
    MGLevel* lev = nullptr;             // device copy of host_lev
    std::vector<MGTop> host_top;        // [run]
    MGTop* top = nullptr;               // device copy
    int* nlev_dev = nullptr;            // [nruns]
    double* red = nullptr;              // [nruns][RED_BLOCKS][2] partial norms
    double* bnorm = nullptr;            // [nruns]
    int* done = nullptr;                // [nruns] converged flags
    int* host_done = nullptr;           // pinned copy
    double* tol = nullptr;              // [nruns]
    int max_cycles = 60;
    int max_nodes0 = 0;                 // largest level-0 node count
    float** inv = nullptr;              // [nruns] inverse of the coarsest operator (transposed), or null
    // work lists of the per-cycle kernels: (run, first item) of each block,
    // for every level l the runs whose tail level lies below l
    int2* tasks = nullptr;              // device copy of all lists
    int coarse_off[MG_MAX_LEVELS] = {}, coarse_len[MG_MAX_LEVELS] = {};   // all nodes of level l + 1
    int tile_off[MG_MAX_LEVELS] = {}, tile_len[MG_MAX_LEVELS] = {};       // smoother tiles of level l
    // levels from tail_lev[run] down are cycled by one block per run in
    // shared memory (k_mg_tail); the level lists hold only the levels above
    std::vector<int> tail_lev;
    int* tail_lev_dev = nullptr;        // [nruns]
    int max_tail = 0;                   // largest tail_lev over the runs
    size_t tail_smem = 0;               // dynamic shared memory of k_mg_tail
    int threads = 256;                  // threads per block of the level kernels (64..1024, a multiple of 32)
    int max_blocks = 1216;              // cap on blocks per run of the once-per-solve node kernels
};

bool field_grid_ok(int nz, int nr);
// bytes for the runs' grids (cells per run)
size_t field_workspace_bytes(const std::vector<int>& nz, const std::vector<int>& nr);
// phi: the simulation's node potential, runs laid end to end at node_base
int field_init(FieldSolver& fs, const std::vector<pd_config>& cfgs, const std::vector<uint32_t>& node_base,
               double* phi, void* ws, size_t bytes, cudaStream_t s);
void field_free(FieldSolver& fs);
// rho_e + rho_h (fixed point) -> phi (warm-started from its current value) -> E
// for every run; the anode potential of each run is RunState::V.  With
// host_check, cycles run until every run reaches its tolerance (the host
// reads the flags between cycles); otherwise exactly `cycles` cycles are
// issued with no host synchronisation (runs already converged skip them),
// so the solve can be captured in a CUDA graph.  Records relres / cycles.
cudaError_t field_solve(FieldSolver& fs, const long long* rho_e, const long long* rho_h, double* phi, float2* E,
                const RunInfo* runs, RunState* rs, int host_check, int cycles, cudaStream_t s,
                int* kernels = nullptr);   // adds the number of kernels launched

// E = -grad(phi) of every run; flags runs whose solve met a non-finite value
// and folds each run's final residual into RunState::relres_max
void field_efield(FieldSolver& fs, const double* phi, const RunInfo* runs, float2* E, DevState* st, RunState* rs,
                  cudaStream_t s);

// Warm start of the solve (see pd_set_warm_start).  History kept across
// solves, per node (C/m^3 and V) and per run (V):
struct WarmHistory {
    double* rho_last;   // density of the most recent solve
    double* rho_prev;   // density of the solve before it
    double* rho_prev2;  // density of the solve before that
    double* phi_prev;   // potential of the solve before the most recent one
    double* phi_prev2;  // potential of the solve before that
    double* V_last;     // [runs] anode voltage of the most recent solve
    double* V_prev;     // [runs] of the one before
    double* V_prev2;    // [runs] of the one before that
};
// Forms of the learned start: the reference the network's input and the
// base of its output are taken against.
//   absolute: d = rho, base = V z / L
//   delta: d = rho - rho', base = phi' + (V - V') z / L
//   extrapolated: d = rho - (2 rho' - rho''),
//                 base = 2 phi' - phi'' + (V - 2 V' + V'') z / L
enum WarmForm { WARM_ABSOLUTE = 0, WARM_DELTA = 1, WARM_EXTRAP = 2 };
// at the start of every solve: shift the history and record the current
// density (Verboncoeur volumes, halved on the electrode rows) and voltage;
// with `extrapolate`, phi := 2 phi - phi_prev on the interior rows (phi_prev
// taken before the shift)
void warm_history(FieldSolver& fs, const long long* rho_e, const long long* rho_h, const RunInfo* runs,
                  const RunState* rs, double* phi, const WarmHistory& h, bool extrapolate, cudaStream_t s);
// d of the form; rmax[run] = max |d|; x = d / rmax
void warm_inputs(FieldSolver& fs, const WarmHistory& h, int form, const RunInfo* runs, double* rmax, float* x,
                 cudaStream_t s);
// interior rows of phi := base + y rmax dz^2 / eps0 (y = null: the base alone)
void warm_apply(FieldSolver& fs, const float* y, const WarmHistory& h, int form, const RunInfo* runs,
                const RunState* rs, const double* rmax, double* phi, cudaStream_t s);
// training targets t = (phi - base) eps0 / (rmax dz^2) at every node, with
// the voltages of the history (call after a solve)
void warm_targets(FieldSolver& fs, const double* phi, const WarmHistory& h, int form, const RunInfo* runs,
                  const double* rmax, float* t, cudaStream_t s);

}  // namespace pd
