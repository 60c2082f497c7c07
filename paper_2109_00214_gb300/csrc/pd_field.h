// pd_field.h -- Poisson solve (Eq. (8)) and E = -grad(phi) on the r-z node grid.
#pragma once
#include <cstddef>
#include "pd.h"
#include "pd_internal.cuh"

namespace pd {

constexpr int MG_MAX_LEVELS = 12;

struct MGLevel {
    int nz, nr;              // cells
    double dz, dr;
    double *x, *f, *r;       // (nz+1)(nr+1) nodes each
    double *ap, *am, *b;     // per radial node j: radial face and axial coefficients
};

struct FieldSolver {
    int nlev = 0;
    MGLevel lev[MG_MAX_LEVELS];
    double* fv_over_verb = nullptr;   // per radial node: finite-volume / Verboncoeur volume
    double* verb_base = nullptr;      // per radial node: Verboncoeur volume of an interior row
    double* red = nullptr;            // reduction scratch
    double* host_red = nullptr;       // pinned host copy
    double weight = 0, tol = 1e-8, V0 = 0;
    int max_cycles = 60;
    int nz = 0, nr = 0;
};

bool field_grid_ok(int nz, int nr);
size_t field_workspace_bytes(int nz, int nr);
int field_init(FieldSolver& fs, const pd_config& c, void* ws, size_t bytes, cudaStream_t s);
// rho_e + rho_h (fixed point) -> phi (warm-started from its current value) -> E;
// the anode potential is DevState::V.  Records relres / cycles in DevState.
void field_free(FieldSolver& fs);
int field_solve(FieldSolver& fs, const long long* rho_e, const long long* rho_h, double* phi, float2* E,
                DevState* st, cudaStream_t s);

}  // namespace pd
