// pd_field.cu -- Poisson solve of Eq. (8), read as lap(phi) = -rho/eps0, by
// geometric multigrid on the r-z node grid of every run, and E = -grad(phi).
//
// Discretisation (finite volumes around each node (i, j)):
//   ap_j (phi_{j+1} - phi_j) + am_j (phi_{j-1} - phi_j)
//     + b_j (phi_{i+1} - 2 phi_i + phi_{i-1}) = -rho_ij Vfv_j / eps0
// with ap_j = 2 pi r_{j+1/2} dz/dr (0 at r = R), am_j = 2 pi r_{j-1/2} dz/dr (0
// on the axis), b_j = A_j / dz, A_j the area of the node's radial extent and
// Vfv_j = A_j dz.  The node density rho_ij = Q_ij / V_ij uses Verboncoeur's
// volumes.  phi = 0 on the cathode row, V on the anode row.
//
// Multigrid: V(2,2) cycles with red-black Gauss-Seidel, residual restriction
// by full weighting of the integrated residuals (weights 1, 1/2, 1/4),
// bilinear prolongation, coefficients rediscretised on each level, and an
// exact solve on the coarsest level: the inverse of its operator, formed on
// the host once, applied by one block (Gauss-Seidel sweeps instead when the
// coarsest level has more than MG_DIRECT_MAX unknowns).  Double precision.
//
// Batched over runs: each level operation is one launch with blockIdx.y = run
// (runs of different sizes and depths; a block whose run has no such level,
// or has converged, returns at once).  Per-run residual norms and converged
// flags stay on the device.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pd_field.h"

namespace pd {

namespace {
constexpr double QE_ = 1.602176634e-19;
constexpr double EPS0_ = 8.8541878128e-12;
constexpr double PI_ = 3.14159265358979323846;
constexpr int RED_BLOCKS = 64;
constexpr int MAP_CHUNK = 256;      // items of one work-list entry

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

void level_dims(int nz, int nr, int* nzs, int* nrs, int& nlev) {
    nzs[0] = nz;
    nrs[0] = nr;
    nlev = 1;
    while (nlev < MG_MAX_LEVELS && nzs[nlev - 1] % 2 == 0 && nrs[nlev - 1] % 2 == 0 && nzs[nlev - 1] > 8 &&
           nrs[nlev - 1] > 8) {
        nzs[nlev] = nzs[nlev - 1] / 2;
        nrs[nlev] = nrs[nlev - 1] / 2;
        ++nlev;
    }
}

// unknowns of the coarsest level (interior rows, all radial nodes)
int coarse_unknowns(const int* a, const int* b, int n) { return (a[n - 1] - 1) * (b[n - 1] + 1); }

constexpr int SP_TI = 8, SP_TJ = 32;   // smoother tile: interior rows x radial nodes

int chunks(long long n) { return (int)((n + MAP_CHUNK - 1) / MAP_CHUNK); }
int tiles_of(int nz, int nr) { return ((nz - 1 + SP_TI - 1) / SP_TI) * ((nr + 1 + SP_TJ - 1) / SP_TJ); }

// work-list entries of one run (all levels that smooth)
size_t run_tasks(int nz, int nr) {
    int a[MG_MAX_LEVELS], b[MG_MAX_LEVELS], n;
    level_dims(nz, nr, a, b, n);
    size_t t = 0;
    for (int l = 0; l + 1 < n; ++l)
        t += chunks((long long)(a[l] - 1) * (b[l] + 1)) + chunks((long long)(a[l + 1] + 1) * (b[l + 1] + 1)) +
             tiles_of(a[l], b[l]);
    return t;
}

size_t run_bytes(int nz, int nr) {
    int a[MG_MAX_LEVELS], b[MG_MAX_LEVELS], n;
    level_dims(nz, nr, a, b, n);
    size_t t = 0;
    for (int l = 0; l < n; ++l) {
        const size_t nodes = (size_t)(a[l] + 1) * (b[l] + 1);
        t += 4 * al(nodes * 8) + 3 * al((size_t)(b[l] + 1) * 8);
    }
    const size_t m = (size_t)coarse_unknowns(a, b, n);
    if (m <= (size_t)MG_DIRECT_MAX) t += al(m * m * 8);
    return t + 2 * al((size_t)(nr + 1) * 8);
}
}  // namespace

bool field_grid_ok(int nz, int nr) {
    int a[MG_MAX_LEVELS], b[MG_MAX_LEVELS], n;
    level_dims(nz, nr, a, b, n);
    return (a[n - 1] + 1) * (b[n - 1] + 1) <= 1024 && a[n - 1] >= 2 && b[n - 1] >= 2;
}

size_t field_workspace_bytes(const std::vector<int>& nz, const std::vector<int>& nr) {
    size_t t = 0;
    const size_t R = nz.size();
    size_t tasks = 0;
    for (size_t r = 0; r < R; ++r) {
        t += run_bytes(nz[r], nr[r]);
        tasks += run_tasks(nz[r], nr[r]);
    }
    t += al(tasks * sizeof(int2) + 8);
    t += al(R * MG_MAX_LEVELS * sizeof(MGLevel)) + al(R * 4) * 3 + al(R * RED_BLOCKS * 2 * 8) + al(R * 8) * 2 +
         al(R * 16) + al(R * sizeof(double*));
    return t;
}

// ------------------------------------------------------------------
// kernels (blockIdx.y = run)
// ------------------------------------------------------------------
__device__ __forceinline__ bool level_active(const int* nlev, const int* done, int r, int l, bool coarsest) {
    if (done && done[r]) return false;
    const int n = nlev[r];
    return coarsest ? (l == n - 1) : (l < n - 1);
}

__global__ void k_rhs(const long long* rho_e, const long long* rho_h, const double* fv_over_verb,
                      const double* verb_base, const int* fvb_off, const MGLevel* lev, const RunInfo* runs,
                      const RunState* rs, double* phi) {
    const int run = blockIdx.y;
    const MGLevel L = lev[run * MG_MAX_LEVELS];
    const RunInfo& RI = runs[run];
    const int W = L.nr + 1;
    const int n = (L.nz + 1) * W;
    const double V = rs[run].V;
    const double qw = QE_ * RI.weight / 4294967296.0;
    const int fo = fvb_off[run];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = k / W, j = k - i * W;
        const uint32_t g = RI.node_base + (uint32_t)k;
        if (i == 0) {
            phi[g] = 0.0;
            L.f[k] = 0.0;
            continue;
        }
        if (i == L.nz) {
            phi[g] = V;
            L.f[k] = 0.0;
            continue;
        }
        // rho_ij (C/m^3) = q W rho_int 2^-32 / V_verb; rhs = rho Vfv / eps0
        const double rho = qw * (double)(rho_e[g] + rho_h[g]) / verb_base[fo + j];
        double v = rho * (fv_over_verb[fo + j] * verb_base[fo + j]) / EPS0_;
        if (i == L.nz - 1) v += L.b[j] * V;
        L.f[k] = v;
    }
}

__device__ __forceinline__ double apply_A(const MGLevel& L, const double* x, int i, int j) {
    const int W = L.nr + 1;
    const int k = i * W + j;
    double s = (L.ap[j] + L.am[j] + 2.0 * L.b[j]) * x[k];
    if (j < L.nr) s -= L.ap[j] * x[k + 1];
    if (j > 0) s -= L.am[j] * x[k - 1];
    if (i + 1 < L.nz) s -= L.b[j] * x[k + W];
    if (i - 1 > 0) s -= L.b[j] * x[k - W];
    return s;
}

// red-black Gauss-Seidel on the interior rows (Dirichlet neighbours are part
// of f on level 0 and zero for the corrections): see k_smooth_pair

// Two half-sweeps of red-black Gauss-Seidel in one launch: color c1 on a
// tile and the ring of nodes around it, then color c2 on the tile, in shared
// memory; reads `src`, writes the tile's interior-row nodes to `dst` (so no
// block reads a value another block has already updated: the same result as
// two separate half-sweeps).  Tile: SP_TI interior rows x SP_TJ radial nodes;
// the work list gives each block its (run, tile).
__global__ void __launch_bounds__(256) k_smooth_pair(const MGLevel* lev, const int* done, int l, int c1, int swap,
                                                     const int2* tasks) {
    __shared__ double xs[SP_TI + 4][SP_TJ + 4];
    __shared__ double fsm[SP_TI + 2][SP_TJ + 2];
    __shared__ double cap[SP_TJ + 2], cam[SP_TJ + 2], cb[SP_TJ + 2];
    const int2 tk = tasks[blockIdx.x];
    const int run = tk.x;
    if (done[run]) return;
    const MGLevel L = lev[run * MG_MAX_LEVELS + l];
    const double* src = swap ? L.x2 : L.x;
    double* dst = swap ? L.x : L.x2;
    const int W = L.nr + 1;
    const int tj = (W + SP_TJ - 1) / SP_TJ;
    const int i0 = 1 + (tk.y / tj) * SP_TI, j0 = (tk.y % tj) * SP_TJ;
    for (int q = threadIdx.x; q < (SP_TI + 4) * (SP_TJ + 4); q += blockDim.x) {
        const int a = q / (SP_TJ + 4), c = q % (SP_TJ + 4);
        const int i = i0 - 2 + a, j = j0 - 2 + c;
        // only interior rows are read by the update (Dirichlet rows enter through f)
        xs[a][c] = (i >= 1 && i <= L.nz - 1 && j >= 0 && j <= L.nr) ? src[i * W + j] : 0.0;
    }
    for (int q = threadIdx.x; q < (SP_TI + 2) * (SP_TJ + 2); q += blockDim.x) {
        const int a = q / (SP_TJ + 2), c = q % (SP_TJ + 2);
        const int i = i0 - 1 + a, j = j0 - 1 + c;
        fsm[a][c] = (i >= 1 && i <= L.nz - 1 && j >= 0 && j <= L.nr) ? L.f[i * W + j] : 0.0;
    }
    for (int c = threadIdx.x; c < SP_TJ + 2; c += blockDim.x) {
        const int j = j0 - 1 + c;
        const bool in = j >= 0 && j <= L.nr;
        cap[c] = in ? L.ap[j] : 0.0;
        cam[c] = in ? L.am[j] : 0.0;
        cb[c] = in ? L.b[j] : 0.0;
    }
    __syncthreads();
    // node (i, j) of shared row a = i - i0 + 2, column c = j - j0 + 2
    auto update = [&](int i, int j) {
        const int a = i - i0 + 2, c = j - j0 + 2, cc = c - 1;
        double s = fsm[a - 1][c - 1];
        if (j < L.nr) s += cap[cc] * xs[a][c + 1];
        if (j > 0) s += cam[cc] * xs[a][c - 1];
        if (i + 1 < L.nz) s += cb[cc] * xs[a + 1][c];
        if (i - 1 > 0) s += cb[cc] * xs[a - 1][c];
        xs[a][c] = s / (cap[cc] + cam[cc] + 2.0 * cb[cc]);
    };
    for (int q = threadIdx.x; q < (SP_TI + 2) * (SP_TJ + 2); q += blockDim.x) {
        const int i = i0 - 1 + q / (SP_TJ + 2), j = j0 - 1 + q % (SP_TJ + 2);
        if (i >= 1 && i <= L.nz - 1 && j >= 0 && j <= L.nr && ((i + j) & 1) == c1) update(i, j);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < SP_TI * SP_TJ; q += blockDim.x) {
        const int i = i0 + q / SP_TJ, j = j0 + q % SP_TJ;
        if (i <= L.nz - 1 && j <= L.nr && ((i + j) & 1) != c1) update(i, j);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < SP_TI * SP_TJ; q += blockDim.x) {
        const int i = i0 + q / SP_TJ, j = j0 + q % SP_TJ;
        if (i <= L.nz - 1 && j <= L.nr) dst[i * W + j] = xs[i - i0 + 2][j - j0 + 2];
    }
}

// residual of level l; with `red`, per-block partial sums of r^2 and f^2
__global__ void k_residual(const MGLevel* lev, const int* nlev, const int* done, int l, double* red) {
    const int run = blockIdx.y;
    const bool act = red ? (nlev[run] > 0) : level_active(nlev, done, run, l, false);
    double acc = 0.0, accb = 0.0;
    if (act) {
        const MGLevel L = lev[run * MG_MAX_LEVELS + l];
        const int W = L.nr + 1;
        const int n = (L.nz - 1) * W;
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
            const int i = 1 + q / W, j = q - (i - 1) * W;
            const int k = i * W + j;
            const double r = L.f[k] - apply_A(L, L.x, i, j);
            L.r[k] = r;
            acc += r * r;
            accb += L.f[k] * L.f[k];
        }
    }
    if (red) {
        for (int o = 16; o > 0; o >>= 1) {
            acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
            accb += __shfl_down_sync(0xFFFFFFFFu, accb, o);
        }
        __shared__ double sa[32], sb[32];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) {
            sa[w] = acc;
            sb[w] = accb;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0, tb = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                t += sa[q];
                tb += sb[q];
            }
            red[(run * RED_BLOCKS + blockIdx.x) * 2] = t;
            red[(run * RED_BLOCKS + blockIdx.x) * 2 + 1] = tb;
        }
    }
}

// residual of level l on the interior rows (work list of the level)
__global__ void k_residual_tasks(const MGLevel* lev, const int* done, int l, const int2* tasks) {
    const int2 tk = tasks[blockIdx.x];
    const int run = tk.x;
    if (done[run]) return;
    const MGLevel L = lev[run * MG_MAX_LEVELS + l];
    const int W = L.nr + 1;
    const int n = min((L.nz - 1) * W, tk.y + MAP_CHUNK);
    for (int q = tk.y + threadIdx.x; q < n; q += blockDim.x) {
        const int i = 1 + q / W, j = q - (i - 1) * W;
        const int k = i * W + j;
        L.r[k] = L.f[k] - apply_A(L, L.x, i, j);
    }
}

// per run: relres = |r| / |b|, converged flag, bookkeeping
__global__ void k_norms(const double* red, double* bnorm, int* done, const double* tol, RunState* rs, int nruns,
                        int cycle, int first) {
    const int run = blockIdx.x * blockDim.x + threadIdx.x;
    if (run >= nruns) return;
    double a = 0, b = 0;
    for (int q = 0; q < RED_BLOCKS; ++q) {
        a += red[(run * RED_BLOCKS + q) * 2];
        b += red[(run * RED_BLOCKS + q) * 2 + 1];
    }
    const double rn = sqrt(a), bn = sqrt(b);
    if (first) done[run] = 0;
    if (done[run]) return;
    bnorm[run] = bn;
    const double rel = bn > 0 ? rn / bn : 0.0;
    rs[run].relres = rel;
    rs[run].cycles = (double)cycle;
    if (!(rel == rel) || !(bn == bn)) {
        done[run] = 2;              // non-finite: stop this run
        return;
    }
    if (bn == 0.0 || rel <= tol[run]) done[run] = 1;
}

// coarse rhs = sum of the fine integrated residuals over the coarse control
// volume (full weighting scaled by 4); zero initial coarse correction
__global__ void k_restrict(const MGLevel* lev, const int* done, int l, const int2* tasks) {
    const int2 tk = tasks[blockIdx.x];
    const int run = tk.x;
    if (done[run]) return;
    const MGLevel F = lev[run * MG_MAX_LEVELS + l];
    const MGLevel Cl = lev[run * MG_MAX_LEVELS + l + 1];
    const int Wc = Cl.nr + 1, Wf = F.nr + 1;
    const int n = min((Cl.nz + 1) * Wc, tk.y + MAP_CHUNK);
    for (int k = tk.y + threadIdx.x; k < n; k += blockDim.x) {
        const int I = k / Wc, J = k - I * Wc;
        Cl.x[k] = 0.0;
        if (I == 0 || I == Cl.nz) {
            Cl.f[k] = 0.0;
            continue;
        }
        double s = 0.0;
        for (int di = -1; di <= 1; ++di) {
            const int i = 2 * I + di;
            if (i <= 0 || i >= F.nz) continue;
            const double wi = di == 0 ? 1.0 : 0.5;
            for (int dj = -1; dj <= 1; ++dj) {
                const int j = 2 * J + dj;
                if (j < 0 || j > F.nr) continue;
                const double wj = dj == 0 ? 1.0 : 0.5;
                s += wi * wj * F.r[i * Wf + j];
            }
        }
        Cl.f[k] = s;
    }
}

__global__ void k_prolong(const MGLevel* lev, const int* done, int l, const int2* tasks) {
    const int2 tk = tasks[blockIdx.x];
    const int run = tk.x;
    if (done[run]) return;
    const MGLevel F = lev[run * MG_MAX_LEVELS + l];
    const MGLevel Cl = lev[run * MG_MAX_LEVELS + l + 1];
    const int Wc = Cl.nr + 1, Wf = F.nr + 1;
    const int n = min((F.nz - 1) * Wf, tk.y + MAP_CHUNK);
    for (int q = tk.y + threadIdx.x; q < n; q += blockDim.x) {
        const int i = 1 + q / Wf, j = q - (i - 1) * Wf;
        const int I0 = i >> 1, J0 = j >> 1;
        const int I1 = (i & 1) ? I0 + 1 : I0, J1 = (j & 1) ? J0 + 1 : J0;
        const double c = 0.25 * (Cl.x[I0 * Wc + J0] + Cl.x[I1 * Wc + J0] + Cl.x[I0 * Wc + J1] + Cl.x[I1 * Wc + J1]);
        F.x[i * Wf + j] += c;
    }
}

// coarsest level of each run whose hierarchy ends at level l (blockIdx.x =
// run): x = A^-1 f with the stored inverse (transposed: column v of A^-1 at
// inv[v * m]), or Gauss-Seidel sweeps when the run has none
__global__ void __launch_bounds__(256) k_coarse(const MGLevel* lev, const int* nlev, const int* done,
                                                const double* const* inv, int l, int sweeps) {
    const int run = blockIdx.x;
    if (!level_active(nlev, done, run, l, true)) return;
    const MGLevel L = lev[run * MG_MAX_LEVELS + l];
    const int W = L.nr + 1;
    const int n = (L.nz - 1) * W;
    const double* Ai = inv[run];
    if (Ai) {
        __shared__ double f[MG_DIRECT_MAX];
        for (int q = threadIdx.x; q < n; q += blockDim.x) f[q] = L.f[W + q];
        __syncthreads();
        for (int u = threadIdx.x; u < n; u += blockDim.x) {
            double acc = 0.0;
            for (int v = 0; v < n; ++v) acc += Ai[(size_t)v * n + u] * f[v];
            L.x[W + u] = acc;
        }
        return;
    }
    for (int it = 0; it < sweeps; ++it) {
        for (int color = 0; color < 2; ++color) {
            for (int q = threadIdx.x; q < n; q += blockDim.x) {
                const int i = 1 + q / W, j = q - (i - 1) * W;
                if (((i + j) & 1) != color) continue;
                const int k = i * W + j;
                double s = L.f[k];
                if (j < L.nr) s += L.ap[j] * L.x[k + 1];
                if (j > 0) s += L.am[j] * L.x[k - 1];
                if (i + 1 < L.nz) s += L.b[j] * L.x[k + W];
                if (i - 1 > 0) s += L.b[j] * L.x[k - W];
                L.x[k] = s / (L.ap[j] + L.am[j] + 2.0 * L.b[j]);
            }
            __syncthreads();
        }
    }
}

// E = -grad(phi): central inside, one-sided at the electrodes, E_r = 0 on the
// axis and at r = R
__global__ void k_efield(const double* phi, const RunInfo* runs, const double* dzr, float2* E) {
    const int run = blockIdx.y;
    const RunInfo& RI = runs[run];
    const int nz = RI.nz, nr = RI.nr;
    const double dz = dzr[2 * run], dr = dzr[2 * run + 1];
    const int W = nr + 1;
    const int n = (nz + 1) * W;
    const double* p = phi + RI.node_base;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = k / W, j = k - i * W;
        double ez, er;
        if (i == 0) ez = -(p[k + W] - p[k]) / dz;
        else if (i == nz) ez = -(p[k] - p[k - W]) / dz;
        else ez = -(p[k + W] - p[k - W]) / (2.0 * dz);
        if (j == 0 || j == nr) er = 0.0;
        else er = -(p[k + 1] - p[k - 1]) / (2.0 * dr);
        E[RI.node_base + k] = make_float2((float)ez, (float)er);
    }
}

__global__ void k_solve_epilogue(const int* done, int nruns, DevState* st, RunState* rs) {
    for (int r = threadIdx.x; r < nruns; r += blockDim.x) {
        if (done[r] == 2) atomicOr(&st->error, ERR_NONFINITE);
        const double rel = rs[r].relres;
        if (!(rel <= rs[r].relres_max)) rs[r].relres_max = rel;   // NaN propagates
    }
}

// ------------------------------------------------------------------
// host
// ------------------------------------------------------------------
static int blocks_for(const FieldSolver& fs, int n) {
    int b = (n + fs.threads - 1) / fs.threads;
    return b < 1 ? 1 : (b > fs.max_blocks ? fs.max_blocks : b);
}

// Inverse of the coarsest operator by Gauss-Jordan elimination with partial
// pivoting; unknown u = (i - 1) (nr + 1) + j for interior rows i and radial
// nodes j, the rows of the smoother's equation.  Stored transposed.
static bool invert_coarse(int nz, int nr, const std::vector<double>& ap, const std::vector<double>& am,
                          const std::vector<double>& bb, std::vector<double>& out) {
    const int W = nr + 1, m = (nz - 1) * W;
    std::vector<double> A((size_t)m * m, 0.0), X((size_t)m * m, 0.0);
    for (int u = 0; u < m; ++u) {
        const int i = 1 + u / W, j = u % W;
        A[(size_t)u * m + u] = ap[j] + am[j] + 2.0 * bb[j];
        if (j < nr) A[(size_t)u * m + u + 1] = -ap[j];
        if (j > 0) A[(size_t)u * m + u - 1] = -am[j];
        if (i + 1 < nz) A[(size_t)u * m + u + W] = -bb[j];
        if (i - 1 > 0) A[(size_t)u * m + u - W] = -bb[j];
        X[(size_t)u * m + u] = 1.0;
    }
    for (int c = 0; c < m; ++c) {
        int p = c;
        for (int r = c + 1; r < m; ++r)
            if (std::fabs(A[(size_t)r * m + c]) > std::fabs(A[(size_t)p * m + c])) p = r;
        if (!(std::fabs(A[(size_t)p * m + c]) > 0.0)) return false;
        if (p != c)
            for (int k = 0; k < m; ++k) {
                std::swap(A[(size_t)p * m + k], A[(size_t)c * m + k]);
                std::swap(X[(size_t)p * m + k], X[(size_t)c * m + k]);
            }
        const double d = A[(size_t)c * m + c];
        for (int k = 0; k < m; ++k) {
            A[(size_t)c * m + k] /= d;
            X[(size_t)c * m + k] /= d;
        }
        for (int r = 0; r < m; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * m + c];
            if (f == 0.0) continue;
            for (int k = 0; k < m; ++k) {
                A[(size_t)r * m + k] -= f * A[(size_t)c * m + k];
                X[(size_t)r * m + k] -= f * X[(size_t)c * m + k];
            }
        }
    }
    out.assign((size_t)m * m, 0.0);
    for (int u = 0; u < m; ++u)
        for (int v = 0; v < m; ++v) out[(size_t)v * m + u] = X[(size_t)u * m + v];
    return true;
}

int field_init(FieldSolver& fs, const std::vector<pd_config>& cfgs, const std::vector<uint32_t>& node_base,
               double* phi, void* ws, size_t bytes, cudaStream_t s) {
    const int R = (int)cfgs.size();
    {
        std::vector<int> nz(R), nr(R);
        for (int r = 0; r < R; ++r) {
            nz[r] = cfgs[r].nz;
            nr[r] = cfgs[r].nr;
        }
        if (field_workspace_bytes(nz, nr) > bytes) return 1;   // checked before anything is written
    }
    char* w = (char*)ws;
    size_t o = 0;
    auto take = [&](size_t sz) {
        char* p = w + o;
        o += al(sz);
        return p;
    };
    fs.nruns = R;
    fs.nlev.assign(R, 0);
    fs.host_lev.assign((size_t)R * MG_MAX_LEVELS, MGLevel{});
    fs.max_levels = 0;
    fs.max_nodes0 = 0;
    fs.max_cycles = cfgs[0].poisson_max_cycles > 0 ? cfgs[0].poisson_max_cycles : 60;
    std::vector<double> fvv_all, vb_all, tol(R), dzr(2 * (size_t)R);
    std::vector<int> fvb_off(R);
    std::vector<double*> inv(R, nullptr);
    for (int r = 0; r < R; ++r) {
        const pd_config& c = cfgs[r];
        int a[MG_MAX_LEVELS], b[MG_MAX_LEVELS], n;
        level_dims(c.nz, c.nr, a, b, n);
        fs.nlev[r] = n;
        fs.max_levels = std::max(fs.max_levels, n);
        fs.max_nodes0 = std::max(fs.max_nodes0, (c.nz + 1) * (c.nr + 1));
        tol[r] = c.poisson_tol;
        dzr[2 * r] = c.dz;
        dzr[2 * r + 1] = c.dr;
        for (int l = 0; l < n; ++l) {
            MGLevel& L = fs.host_lev[(size_t)r * MG_MAX_LEVELS + l];
            L.nz = a[l];
            L.nr = b[l];
            const double dz = c.dz * (double)(1 << l), dr = c.dr * (double)(1 << l);
            const size_t nodes = (size_t)(L.nz + 1) * (L.nr + 1);
            L.x = l == 0 ? phi + node_base[r] : (double*)take(nodes * 8);
            L.f = (double*)take(nodes * 8);
            L.r = (double*)take(nodes * 8);
            L.x2 = (double*)take(nodes * 8);
            L.ap = (double*)take((size_t)(L.nr + 1) * 8);
            L.am = (double*)take((size_t)(L.nr + 1) * 8);
            L.b = (double*)take((size_t)(L.nr + 1) * 8);
            std::vector<double> ap(L.nr + 1), am(L.nr + 1), bb(L.nr + 1);
            const double Rr = L.nr * dr;
            for (int j = 0; j <= L.nr; ++j) {
                const double rp = (j + 0.5) * dr, rm = (j - 0.5) * dr;
                ap[j] = j < L.nr ? 2.0 * PI_ * rp * dz / dr : 0.0;
                am[j] = j > 0 ? 2.0 * PI_ * rm * dz / dr : 0.0;
                double A;
                if (j == 0) A = PI_ * (0.5 * dr) * (0.5 * dr);
                else if (j == L.nr) A = PI_ * (Rr * Rr - (Rr - 0.5 * dr) * (Rr - 0.5 * dr));
                else A = 2.0 * PI_ * j * dr * dr;
                bb[j] = A / dz;
            }
            if (l == n - 1 && coarse_unknowns(a, b, n) <= MG_DIRECT_MAX) {
                const int m = coarse_unknowns(a, b, n);
                std::vector<double> Ai;
                if (!invert_coarse(L.nz, L.nr, ap, am, bb, Ai)) return 1;
                inv[r] = (double*)take((size_t)m * m * 8);
                cudaMemcpyAsync(inv[r], Ai.data(), Ai.size() * 8, cudaMemcpyHostToDevice, s);
            }
            cudaMemcpyAsync(L.ap, ap.data(), ap.size() * 8, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(L.am, am.data(), am.size() * 8, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(L.b, bb.data(), bb.size() * 8, cudaMemcpyHostToDevice, s);
            if (l > 0) cudaMemsetAsync(L.x, 0, nodes * 8, s);
            if (l == 0) {
                fvb_off[r] = (int)fvv_all.size();
                for (int j = 0; j <= L.nr; ++j) {
                    double verb;
                    if (j == 0) verb = PI_ * c.dz * c.dr * c.dr / 3.0;
                    else if (j == c.nr) verb = 2.0 * PI_ * c.dz * c.dr * c.dr * ((double)c.nr / 2.0 - 1.0 / 6.0);
                    else verb = 2.0 * PI_ * c.dz * c.dr * c.dr * (double)j;
                    const double A = bb[j] * dz;      // radial extent area of the control volume
                    vb_all.push_back(verb);
                    fvv_all.push_back(A * dz / verb);  // Vfv / Vverb, Vfv = A dz
                }
            }
        }
    }
    fs.fv_over_verb = (double*)take(fvv_all.size() * 8);
    fs.verb_base = (double*)take(vb_all.size() * 8);
    fs.lev = (MGLevel*)take((size_t)R * MG_MAX_LEVELS * sizeof(MGLevel));
    fs.nlev_dev = (int*)take((size_t)R * 4);
    fs.fvb_off = (int*)take((size_t)R * 4);
    fs.done = (int*)take((size_t)R * 4);
    fs.red = (double*)take((size_t)R * RED_BLOCKS * 2 * 8);
    fs.bnorm = (double*)take((size_t)R * 8);
    fs.tol = (double*)take((size_t)R * 8);
    fs.dzr = (double*)take((size_t)R * 16);
    fs.inv = (double**)take((size_t)R * sizeof(double*));
    // work lists, level by level
    std::vector<int2> tasks;
    for (int l = 0; l < MG_MAX_LEVELS; ++l) {
        auto add = [&](int r, long long n, int step) {
            for (long long q = 0; q < n; q += step) tasks.push_back(make_int2(r, (int)q));
        };
        fs.fine_off[l] = (int)tasks.size();
        for (int r = 0; r < R; ++r)
            if (l + 1 < fs.nlev[r]) {
                const MGLevel& L = fs.host_lev[(size_t)r * MG_MAX_LEVELS + l];
                add(r, (long long)(L.nz - 1) * (L.nr + 1), MAP_CHUNK);
            }
        fs.fine_len[l] = (int)tasks.size() - fs.fine_off[l];
        fs.coarse_off[l] = (int)tasks.size();
        for (int r = 0; r < R; ++r)
            if (l + 1 < fs.nlev[r]) {
                const MGLevel& C = fs.host_lev[(size_t)r * MG_MAX_LEVELS + l + 1];
                add(r, (long long)(C.nz + 1) * (C.nr + 1), MAP_CHUNK);
            }
        fs.coarse_len[l] = (int)tasks.size() - fs.coarse_off[l];
        fs.tile_off[l] = (int)tasks.size();
        for (int r = 0; r < R; ++r)
            if (l + 1 < fs.nlev[r]) {
                const MGLevel& L = fs.host_lev[(size_t)r * MG_MAX_LEVELS + l];
                add(r, tiles_of(L.nz, L.nr), 1);
            }
        fs.tile_len[l] = (int)tasks.size() - fs.tile_off[l];
    }
    fs.tasks = (int2*)take(tasks.size() * sizeof(int2) + 8);
    if (o > bytes) return 1;
    cudaMemcpyAsync(fs.tasks, tasks.data(), tasks.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(fs.inv, inv.data(), (size_t)R * sizeof(double*), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(fs.dzr, dzr.data(), (size_t)R * 16, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(fs.fv_over_verb, fvv_all.data(), fvv_all.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(fs.verb_base, vb_all.data(), vb_all.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(fs.lev, fs.host_lev.data(), fs.host_lev.size() * sizeof(MGLevel), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(fs.nlev_dev, fs.nlev.data(), (size_t)R * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(fs.fvb_off, fvb_off.data(), (size_t)R * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(fs.tol, tol.data(), (size_t)R * 8, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(fs.done, 0, (size_t)R * 4, s);
    if (!fs.host_done && cudaMallocHost(&fs.host_done, (size_t)R * 4) != cudaSuccess) return 1;
    return cudaStreamSynchronize(s) == cudaSuccess ? 0 : 1;
}

void field_free(FieldSolver& fs) {
    if (fs.host_done) cudaFreeHost(fs.host_done);
    fs.host_done = nullptr;
}


// two red-black iterations (four half-sweeps) in two fused launches; the
// second returns the values to x
static int smooth2(FieldSolver& fs, int l, int c1, cudaStream_t s) {
    if (!fs.tile_len[l]) return 0;
    const int2* t = fs.tasks + fs.tile_off[l];
    k_smooth_pair<<<fs.tile_len[l], 256, 0, s>>>(fs.lev, fs.done, l, c1, 0, t);
    k_smooth_pair<<<fs.tile_len[l], 256, 0, s>>>(fs.lev, fs.done, l, c1, 1, t);
    return 2;
}

// one V-cycle of every run that has not converged; returns the kernels launched
static int vcycle(FieldSolver& fs, cudaStream_t s) {
    const int R = fs.nruns;
    const int th = fs.threads;
    int nk = 0;
    // down: smooth, residual, restrict; the coarsest level of each run is solved directly
    for (int l = 0; l < fs.max_levels; ++l) {
        nk += smooth2(fs, l, 0, s);
        if (fs.fine_len[l]) {
            k_residual_tasks<<<fs.fine_len[l], th, 0, s>>>(fs.lev, fs.done, l, fs.tasks + fs.fine_off[l]);
            k_restrict<<<fs.coarse_len[l], th, 0, s>>>(fs.lev, fs.done, l, fs.tasks + fs.coarse_off[l]);
            nk += 2;
        }
        k_coarse<<<R, 256, 0, s>>>(fs.lev, fs.nlev_dev, fs.done, fs.inv, l, 200);
        ++nk;
    }
    // up: prolong, smooth
    for (int l = fs.max_levels - 2; l >= 0; --l) {
        if (!fs.fine_len[l]) continue;
        k_prolong<<<fs.fine_len[l], th, 0, s>>>(fs.lev, fs.done, l, fs.tasks + fs.fine_off[l]);
        ++nk;
        nk += smooth2(fs, l, 1, s);
    }
    return nk;
}

static void norms(FieldSolver& fs, RunState* rs, int cycle, int first, cudaStream_t s) {
    const int R = fs.nruns;
    const dim3 g(RED_BLOCKS, R);
    // fixed shape: the summation order of the norms (and so the cycle count)
    // does not depend on the tuned block size
    k_residual<<<g, 256, 0, s>>>(fs.lev, fs.nlev_dev, nullptr, 0, fs.red);
    k_norms<<<(R + 127) / 128, 128, 0, s>>>(fs.red, fs.bnorm, fs.done, fs.tol, rs, R, cycle, first);
}

int field_solve(FieldSolver& fs, const long long* rho_e, const long long* rho_h, double* phi, float2* E,
                const RunInfo* runs, RunState* rs, int host_check, int cycles, cudaStream_t s, int* kernels) {
    (void)E;
    const int R = fs.nruns;
    const dim3 g0(blocks_for(fs, fs.max_nodes0), R);
    k_rhs<<<g0, fs.threads, 0, s>>>(rho_e, rho_h, fs.fv_over_verb, fs.verb_base, fs.fvb_off, fs.lev, runs, rs, phi);
    norms(fs, rs, 0, 1, s);
    if (kernels) *kernels += 3;
    if (host_check) {
        for (int cyc = 1; cyc <= fs.max_cycles; ++cyc) {
            if (cudaMemcpyAsync(fs.host_done, fs.done, (size_t)R * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return 1;
            if (cudaStreamSynchronize(s) != cudaSuccess) return 1;
            bool all = true;
            for (int r = 0; r < R; ++r) all = all && fs.host_done[r] != 0;
            if (all) break;
            const int nk = vcycle(fs, s);
            norms(fs, rs, cyc, 0, s);
            if (kernels) *kernels += nk + 2;
        }
    } else {
        for (int cyc = 1; cyc <= cycles; ++cyc) {
            const int nk = vcycle(fs, s);
            norms(fs, rs, cyc, 0, s);
            if (kernels) *kernels += nk + 2;
        }
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// E for every run (separate so the caller can time it)
void field_efield(FieldSolver& fs, const double* phi, const RunInfo* runs, float2* E, DevState* st, RunState* rs,
                  cudaStream_t s) {
    const dim3 g(blocks_for(fs, fs.max_nodes0), fs.nruns);
    k_efield<<<g, fs.threads, 0, s>>>(phi, runs, fs.dzr, E);
    k_solve_epilogue<<<1, 128, 0, s>>>(fs.done, fs.nruns, st, rs);
}

// ------------------------------------------------------------------
// warm start
// ------------------------------------------------------------------
// node density of the current fixed-point charge (C/m^3)
__device__ __forceinline__ double node_rho(const long long* rho_e, const long long* rho_h, const double* verb_base,
                                           int fo, const RunInfo& RI, int i, int j, uint32_t g) {
    const double qw = QE_ * RI.weight / 4294967296.0;
    double vol = verb_base[fo + j];
    if (i == 0 || i == RI.nz) vol *= 0.5;
    return qw * (double)(rho_e[g] + rho_h[g]) / vol;
}

// history shift at the start of a solve: rho_prev := rho_last, phi_prev :=
// phi, V_prev := V_last; then rho_last := current density, V_last := V
__global__ void k_warm_history(const long long* rho_e, const long long* rho_h, const double* verb_base,
                               const int* fvb_off, const RunInfo* runs, const RunState* rs, const double* phi,
                               WarmHistory h) {
    const int run = blockIdx.y;
    const RunInfo& RI = runs[run];
    const int W = RI.nr + 1, n = (RI.nz + 1) * W;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = k / W, j = k - i * W;
        const uint32_t g = RI.node_base + (uint32_t)k;
        h.rho_prev[g] = h.rho_last[g];
        h.phi_prev[g] = phi[g];
        h.rho_last[g] = node_rho(rho_e, rho_h, verb_base, fvb_off[run], RI, i, j, g);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        h.V_prev[run] = h.V_last[run];
        h.V_last[run] = rs[run].V;
    }
}

// d = rho_last - ref (ref null: 0); rmax[run] = max |d|
__global__ void k_warm_rmax(const double* rho_last, const double* ref, const RunInfo* runs,
                            unsigned long long* rmax_bits) {
    const int run = blockIdx.y;
    const RunInfo& RI = runs[run];
    const int n = (RI.nz + 1) * (RI.nr + 1);
    double m = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t g = RI.node_base + (uint32_t)k;
        m = fmax(m, fabs(rho_last[g] - (ref ? ref[g] : 0.0)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xFFFFFFFFu, m, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(&rmax_bits[run], (unsigned long long)__double_as_longlong(m));
}

__global__ void k_warm_x(const double* rho_last, const double* ref, const RunInfo* runs, const double* rmax,
                         float* x) {
    const int run = blockIdx.y;
    const RunInfo& RI = runs[run];
    const int n = (RI.nz + 1) * (RI.nr + 1);
    const double rm = rmax[run];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t g = RI.node_base + (uint32_t)k;
        x[g] = rm > 0.0 ? (float)((rho_last[g] - (ref ? ref[g] : 0.0)) / rm) : 0.0f;
    }
}

// the potential the prediction is added to: V z / L, or with a reference
// phi_ref + (V - V_ref) z / L
__device__ __forceinline__ double warm_base(const double* phi_ref, double V, double V_ref, uint32_t g, int i,
                                            int nz) {
    return phi_ref ? phi_ref[g] + (V - V_ref) * (double)i / (double)nz : V * (double)i / (double)nz;
}

__global__ void k_warm_apply(const float* y, const RunInfo* runs, const RunState* rs, const double* rmax,
                             const double* dzr, const double* phi_ref, const double* V_ref, double* phi) {
    const int run = blockIdx.y;
    const RunInfo& RI = runs[run];
    const int W = RI.nr + 1, n = (RI.nz - 1) * W;
    const double V = rs[run].V, Vr = V_ref ? V_ref[run] : 0.0, dz = dzr[2 * run];
    const double sc = y ? rmax[run] * dz * dz / EPS0_ : 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int i = 1 + q / W;
        const uint32_t g = RI.node_base + (uint32_t)(W + q);
        const double base = warm_base(phi_ref, V, Vr, g, i, RI.nz);
        phi[g] = y ? base + (double)y[g] * sc : base;
    }
}

__global__ void k_warm_targets(const double* phi, const RunInfo* runs, const double* V_last, const double* rmax,
                               const double* dzr, const double* phi_ref, const double* V_ref, float* t) {
    const int run = blockIdx.y;
    const RunInfo& RI = runs[run];
    const int W = RI.nr + 1, n = (RI.nz + 1) * W;
    const double V = V_last[run], Vr = V_ref ? V_ref[run] : 0.0, dz = dzr[2 * run], rm = rmax[run];
    const double sc = rm > 0.0 ? EPS0_ / (rm * dz * dz) : 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = k / W;
        const uint32_t g = RI.node_base + (uint32_t)k;
        t[g] = (float)((phi[g] - warm_base(phi_ref, V, Vr, g, i, RI.nz)) * sc);
    }
}

void warm_history(FieldSolver& fs, const long long* rho_e, const long long* rho_h, const RunInfo* runs,
                  const RunState* rs, const double* phi, const WarmHistory& h, cudaStream_t s) {
    const dim3 g(blocks_for(fs, fs.max_nodes0), fs.nruns);
    k_warm_history<<<g, fs.threads, 0, s>>>(rho_e, rho_h, fs.verb_base, fs.fvb_off, runs, rs, phi, h);
}

void warm_inputs(FieldSolver& fs, const WarmHistory& h, bool delta, const RunInfo* runs, double* rmax, float* x,
                 cudaStream_t s) {
    const dim3 g(blocks_for(fs, fs.max_nodes0), fs.nruns);
    const double* ref = delta ? h.rho_prev : nullptr;
    cudaMemsetAsync(rmax, 0, (size_t)fs.nruns * 8, s);
    k_warm_rmax<<<g, fs.threads, 0, s>>>(h.rho_last, ref, runs, (unsigned long long*)rmax);
    k_warm_x<<<g, fs.threads, 0, s>>>(h.rho_last, ref, runs, rmax, x);
}

void warm_apply(FieldSolver& fs, const float* y, const WarmHistory& h, bool delta, const RunInfo* runs,
                const RunState* rs, const double* rmax, double* phi, cudaStream_t s) {
    const dim3 g(blocks_for(fs, fs.max_nodes0), fs.nruns);
    k_warm_apply<<<g, fs.threads, 0, s>>>(y, runs, rs, rmax, fs.dzr, delta ? h.phi_prev : nullptr,
                                          delta ? h.V_prev : nullptr, phi);
}

void warm_targets(FieldSolver& fs, const double* phi, const WarmHistory& h, bool delta, const RunInfo* runs,
                  const double* rmax, float* t, cudaStream_t s) {
    const dim3 g(blocks_for(fs, fs.max_nodes0), fs.nruns);
    k_warm_targets<<<g, fs.threads, 0, s>>>(phi, runs, h.V_last, rmax, fs.dzr, delta ? h.phi_prev : nullptr,
                                            delta ? h.V_prev : nullptr, t);
}

}  // namespace pd
