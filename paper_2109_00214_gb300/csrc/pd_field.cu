// pd_field.cu -- Poisson solve of Eq. (8), read as lap(phi) = -rho/eps0, on the
// r-z node grid of every run, and E = -grad(phi).
//
// Discretisation (finite volumes around each node (i, j)):
//   ap_j (phi_{j+1} - phi_j) + am_j (phi_{j-1} - phi_j)
//     + b_j (phi_{i+1} - 2 phi_i + phi_{i-1}) = -rho_ij Vfv_j / eps0
// with ap_j = 2 pi r_{j+1/2} dz/dr (0 at r = R), am_j = 2 pi r_{j-1/2} dz/dr (0
// on the axis), b_j = A_j / dz, A_j the area of the node's radial extent and
// Vfv_j = A_j dz.  The node density rho_ij = Q_ij / V_ij uses Verboncoeur's
// volumes.  phi = 0 on the cathode row, V on the anode row.  In matrix form
// A phi = b on the interior rows.
//
// Solver: defect correction in double precision around a single-precision
// multigrid.  Each cycle takes the residual r = b - A phi in double (with its
// norm, the convergence test), solves A e = r approximately by one float
// V(2,2) cycle from e = 0, and adds e to phi in double.  GB300 does double
// arithmetic at a small fraction of its float rate, so only the residual and
// the update are double; the cycle converges like a double one as long as
// each correction is accurate to a few digits, and phi reaches residuals far
// below float precision.
//
// V-cycle: red-black Gauss-Seidel (four half-sweeps per launch through a
// shared-memory tile), restriction of the integrated residuals by full
// weighting (1, 1/2, 1/4), bilinear prolongation, coefficients rediscretised
// on each level, and an exact solve on the coarsest level by its inverse
// (formed on the host once; Gauss-Seidel sweeps instead when the coarsest
// level has more than MG_DIRECT_MAX unknowns).
//
// Batched over runs: the per-cycle kernels take work lists of (run, tile or
// chunk) per level, so a launch has only blocks with work; a run that has
// converged skips the rest of the cycles.  Per-run residual norms and
// converged flags stay on the device.
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
constexpr int RED_BLOCKS = 256;      // blocks of a run's residual (a fixed shape: the summation order is fixed)
constexpr int MAP_CHUNK = 256;         // items of one work-list entry
constexpr int SP_TI = 32, SP_TJ = 32;  // smoother tile: interior rows x radial nodes
constexpr int SP_H = 4;                // halo: four half-sweeps per launch
constexpr int TAIL_NODES = 34 * 34;    // levels from the first one with at most this many nodes: k_mg_tail
constexpr int TAIL_THREADS = 512;

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

// first level cycled by k_mg_tail (the coarsest level always qualifies: at
// most 1024 nodes)
int tail_level(const int* a, const int* b, int n) {
    for (int l = 0; l < n; ++l)
        if ((a[l] + 1) * (b[l] + 1) <= TAIL_NODES) return l;
    return n - 1;
}

// k_mg_tail's shared memory for one run: e, f, r per node and ap, am, b,
// dinv per radial node of each tail level
size_t tail_floats(const int* a, const int* b, int n) {
    size_t t = 0;
    for (int l = tail_level(a, b, n); l < n; ++l) t += 3 * (size_t)(a[l] + 1) * (b[l] + 1) + 4 * (size_t)(b[l] + 1);
    return t;
}

int chunks(long long n) { return (int)((n + MAP_CHUNK - 1) / MAP_CHUNK); }
int tiles_of(int nz, int nr) { return ((nz - 1 + SP_TI - 1) / SP_TI) * ((nr + 1 + SP_TJ - 1) / SP_TJ); }

// work-list entries of one run (all levels that smooth)
size_t run_tasks(int nz, int nr) {
    int a[MG_MAX_LEVELS], b[MG_MAX_LEVELS], n;
    level_dims(nz, nr, a, b, n);
    size_t t = 0;
    for (int l = 0; l + 1 < n; ++l)
        t += chunks((long long)(a[l + 1] + 1) * (b[l + 1] + 1)) + tiles_of(a[l], b[l]);
    return t;
}

// device bytes of one run, in the order field_init takes them
size_t run_bytes(int nz, int nr) {
    int a[MG_MAX_LEVELS], b[MG_MAX_LEVELS], n;
    level_dims(nz, nr, a, b, n);
    const size_t W0 = (size_t)nr + 1, nodes0 = ((size_t)nz + 1) * W0;
    size_t t = al(nodes0 * 8) + 6 * al(W0 * 8);            // b, and ap, am, b, dg, cr, iv of level 0 in double
    for (int l = 0; l < n; ++l) {
        const size_t W = (size_t)b[l] + 1, nodes = ((size_t)a[l] + 1) * W;
        t += 3 * al(nodes * 4) + 4 * al(W * 4);             // e, e2, f; ap, am, b, dinv in float
    }
    const size_t m = (size_t)coarse_unknowns(a, b, n);
    if (m <= (size_t)MG_DIRECT_MAX) t += al(m * m * 4);
    return t;
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
    t += al(R * MG_MAX_LEVELS * sizeof(MGLevel)) + al(R * sizeof(MGTop)) + al(R * 4) * 3 +
         al(R * RED_BLOCKS * 2 * 8) + al(R * 8) * 2 + al(R * sizeof(float*)) + al(tasks * sizeof(int2) + 8);
    return t;
}

// ------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------
// b (double) and the electrode rows of phi of every run (blockIdx.y = run)
__global__ void k_rhs(const long long* rho_e, const long long* rho_h, const MGTop* top, const RunInfo* runs,
                      const RunState* rs) {
    const int run = blockIdx.y;
    const MGTop T = top[run];
    const uint32_t nb = runs[run].node_base;
    const int W = T.nr + 1;
    const int n = (T.nz + 1) * W;
    const double V = rs[run].V;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = k / W, j = k - i * W;
        if (i == 0 || i == T.nz) {
            T.phi[k] = i == 0 ? 0.0 : V;
            T.bf[k] = 0.0;
            continue;
        }
        double v = (double)(rho_e[nb + k] + rho_h[nb + k]) * T.cr[j];
        if (i == T.nz - 1) v += T.b[j] * V;
        T.bf[k] = v;
    }
}

// (A x)_ij on an interior node of a correction level, float
__device__ __forceinline__ float apply_Af(const MGLevel& L, const float* x, int i, int j) {
    const int W = L.nr + 1;
    const int k = i * W + j;
    float s = (L.ap[j] + L.am[j] + 2.0f * L.b[j]) * x[k];
    if (j < L.nr) s -= L.ap[j] * x[k + 1];
    if (j > 0) s -= L.am[j] * x[k - 1];
    if (i + 1 < L.nz) s -= L.b[j] * x[k + W];
    if (i - 1 > 0) s -= L.b[j] * x[k - W];
    return s;
}

// The residual r = b - A phi of every run in double, per-block partial sums
// of r^2 (and, with with_b, of b^2) for its norm, and the right-hand side of
// the next correction: level 0's f = r (float).
// blockIdx.y = run; block x takes the interior rows x, x + RED_BLOCKS, ...
// with the threads along the row.  A fixed launch shape, so the summation
// order (and the cycle count) never depends on tuning.
__global__ void __launch_bounds__(256) k_residual_norms(const MGTop* top, const MGLevel* lev, const int* nlev,
                                                        double* red, int with_b) {
    const int run = blockIdx.y;
    double acc = 0.0, accb = 0.0;
    if (nlev[run] > 0) {
        const MGTop T = top[run];
        const MGLevel L = lev[run * MG_MAX_LEVELS];
        const int W = T.nr + 1;
        const double* x = T.phi;
        for (int i = 1 + blockIdx.x; i < T.nz; i += RED_BLOCKS) {
            for (int j = threadIdx.x; j < W; j += blockDim.x) {
                const int k = i * W + j;
                const double xp = j < T.nr ? x[k + 1] : 0.0;
                const double xm = j > 0 ? x[k - 1] : 0.0;
                const double xu = i + 1 < T.nz ? x[k + W] : 0.0;     // the anode row is in b
                const double xd = i - 1 > 0 ? x[k - W] : 0.0;
                const double bk = T.bf[k];
                double r = bk - T.dg[j] * x[k];
                r += T.ap[j] * xp;
                r += T.am[j] * xm;
                r += T.b[j] * (xu + xd);
                L.f[k] = (float)r;
                acc += r * r;
                if (with_b) accb += bk * bk;
            }
        }
    }
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
        if (with_b) red[(run * RED_BLOCKS + blockIdx.x) * 2 + 1] = tb;
    }
}

// per run (one warp each): relres = |r| / |b| (|b| from the first call of
// the solve), converged flag, bookkeeping
__global__ void k_norms(const double* red, double* bnorm, int* done, const double* tol, RunState* rs, int nruns,
                        int cycle, int first) {
    const int run = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (run >= nruns) return;
    double a = 0, b = 0;
    for (int q = lane; q < RED_BLOCKS; q += 32) {
        a += red[(run * RED_BLOCKS + q) * 2];
        if (first) b += red[(run * RED_BLOCKS + q) * 2 + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xFFFFFFFFu, a, o);
        b += __shfl_down_sync(0xFFFFFFFFu, b, o);
    }
    if (lane != 0) return;
    const double rn = sqrt(a);
    if (first) {
        done[run] = 0;
        bnorm[run] = sqrt(b);
    }
    if (done[run]) return;
    const double bn = bnorm[run];
    const double rel = bn > 0 ? rn / bn : 0.0;
    rs[run].relres = rel;
    rs[run].cycles = (double)cycle;
    if (first) rs[run].relres0 = rel;
    if (!(rel == rel) || !(bn == bn)) {
        done[run] = 2;              // non-finite: stop this run
        return;
    }
    if (bn == 0.0 || rel <= tol[run]) done[run] = 1;
}

// Four half-sweeps of red-black Gauss-Seidel on A e = f (colors c1, c2, c1,
// c2: two iterations) in one launch, on a tile of SP_TI interior rows x SP_TJ
// radial nodes in shared memory: the k-th half-sweep updates the tile grown
// by 3 - k rings, so the tile's own nodes end exact (the result of four
// separate half-sweeps).  The work list gives each block its (run, tile).
// Pre-smoothing (POST false, colors 0, 1, 0, 1): starts from e = 0 (the
// correction of a level is zero when its cycle begins) and writes e2.
// Post-smoothing (POST true, colors 1, 0, 1, 0): starts from e2 plus the
// bilinear prolongation of level l + 1's correction (its e), and writes e,
// or, with FINAL (level 0), adds the tile to phi.  No block reads what
// another block of the same launch writes.
template <bool POST, bool FINAL>
__global__ void __launch_bounds__(256) k_smooth4(const MGLevel* lev, const MGTop* top, const int* done, int l,
                                                 const int2* tasks) {
    constexpr int XR = SP_TI + 2 * SP_H, XC = SP_TJ + 2 * SP_H, FR = XR - 2, FC = XC - 2;
    __shared__ float xs[XR][XC + 1];
    __shared__ float fsm[FR][FC];
    __shared__ float cap[FC], cam[FC], cb[FC], cd[FC];
    const int2 tk = tasks[blockIdx.x];
    const int run = tk.x;
    if (done[run]) return;
    const int c1 = POST ? 1 : 0;
    const MGLevel L = lev[run * MG_MAX_LEVELS + l];
    const int W = L.nr + 1;
    const int tj = (W + SP_TJ - 1) / SP_TJ;
    const int i0 = 1 + (tk.y / tj) * SP_TI, j0 = (tk.y % tj) * SP_TJ;
    if (POST) {
        const MGLevel Cl = lev[run * MG_MAX_LEVELS + l + 1];
        const int Wc = Cl.nr + 1;
        const float* ce = Cl.e;
        for (int q = threadIdx.x; q < XR * XC; q += blockDim.x) {
            const int a = q / XC, c = q % XC;
            const int i = i0 - SP_H + a, j = j0 - SP_H + c;
            float v = 0.0f;
            // only interior rows are read by the update (the corrections vanish on the electrodes)
            if (i >= 1 && i <= L.nz - 1 && j >= 0 && j <= L.nr) {
                const int I0 = i >> 1, J0 = j >> 1;
                const int I1 = (i & 1) ? I0 + 1 : I0, J1 = (j & 1) ? J0 + 1 : J0;
                const float cc =
                    0.25f * (ce[I0 * Wc + J0] + ce[I1 * Wc + J0] + ce[I0 * Wc + J1] + ce[I1 * Wc + J1]);
                v = L.e2[i * W + j] + cc;
            }
            xs[a][c] = v;
        }
    } else {
        for (int q = threadIdx.x; q < XR * (XC + 1); q += blockDim.x) (&xs[0][0])[q] = 0.0f;
    }
    for (int q = threadIdx.x; q < FR * FC; q += blockDim.x) {
        const int a = q / FC, c = q % FC;
        const int i = i0 - SP_H + 1 + a, j = j0 - SP_H + 1 + c;
        fsm[a][c] = (i >= 1 && i <= L.nz - 1 && j >= 0 && j <= L.nr) ? L.f[i * W + j] : 0.0f;
    }
    for (int c = threadIdx.x; c < FC; c += blockDim.x) {
        const int j = j0 - SP_H + 1 + c;
        const bool in = j >= 0 && j <= L.nr;
        cap[c] = in ? L.ap[j] : 0.0f;
        cam[c] = in ? L.am[j] : 0.0f;
        cb[c] = in ? L.b[j] : 0.0f;
        cd[c] = in ? L.dinv[j] : 0.0f;
    }
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
        const int grow = 3 - k, color = (k & 1) ? 1 - c1 : c1;
        // the nodes of one color: half of each row of the grown tile
        const int rows = SP_TI + 2 * grow, half = (SP_TJ + 2 * grow) / 2;
        for (int q = threadIdx.x; q < rows * half; q += blockDim.x) {
            const int ii = q / half, jj = q - ii * half;
            const int i = i0 - grow + ii;
            const int jf = j0 - grow;                                   // first column of the row
            const int j = jf + 2 * jj + (((i + jf) & 1) != color ? 1 : 0);
            if (i < 1 || i > L.nz - 1 || j < 0 || j > L.nr) continue;
            const int a = i - i0 + SP_H, c = j - j0 + SP_H, fa = a - 1, fc = c - 1;
            float v = fsm[fa][fc];
            if (j < L.nr) v += cap[fc] * xs[a][c + 1];
            if (j > 0) v += cam[fc] * xs[a][c - 1];
            if (i + 1 < L.nz) v += cb[fc] * xs[a + 1][c];
            if (i - 1 > 0) v += cb[fc] * xs[a - 1][c];
            xs[a][c] = v * cd[fc];
        }
        __syncthreads();
    }
    if (FINAL) {
        double* phi = top[run].phi;
        for (int q = threadIdx.x; q < SP_TI * SP_TJ; q += blockDim.x) {
            const int i = i0 + q / SP_TJ, j = j0 + q % SP_TJ;
            if (i <= L.nz - 1 && j <= L.nr) phi[i * W + j] += (double)xs[i - i0 + SP_H][j - j0 + SP_H];
        }
    } else {
        float* out = POST ? L.e : L.e2;
        for (int q = threadIdx.x; q < SP_TI * SP_TJ; q += blockDim.x) {
            const int i = i0 + q / SP_TJ, j = j0 + q % SP_TJ;
            if (i <= L.nz - 1 && j <= L.nr) out[i * W + j] = xs[i - i0 + SP_H][j - j0 + SP_H];
        }
    }
}

// Coarse right-hand side of level l + 1 = the sum of the fine residuals
// r = f - A e2 (e2: level l's pre-smoothed correction, r computed here)
// over the coarse control volume (full weighting scaled by 4); zero coarse
// correction.  Work list of the coarse level's nodes.
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
        if (I == 0 || I == Cl.nz) {
            Cl.f[k] = 0.0f;
            continue;
        }
        float s = 0.0f;
        for (int di = -1; di <= 1; ++di) {
            const int i = 2 * I + di;
            if (i <= 0 || i >= F.nz) continue;
            const float wi = di == 0 ? 1.0f : 0.5f;
            for (int dj = -1; dj <= 1; ++dj) {
                const int j = 2 * J + dj;
                if (j < 0 || j > F.nr) continue;
                const float wj = dj == 0 ? 1.0f : 0.5f;
                s += wi * wj * (F.f[i * Wf + j] - apply_Af(F, F.e2, i, j));
            }
        }
        Cl.f[k] = s;
    }
}

// The levels of one run from its first tail level T down to its coarsest,
// one V(2,2) cycle by one block in shared memory (blockIdx.x = run): the
// per-level kernels' operations in their order -- four red-black half-sweeps
// (colors 0, 1, 0, 1), the residual, the full-weighting restriction, on the
// coarsest level e = A^-1 f with the stored inverse (transposed: column v at
// inv[v * m]) or `sweeps` Gauss-Seidel sweeps, then bilinear prolongation
// and four half-sweeps (colors 1, 0, 1, 0) on the way up.  Input: f of level
// T (its e is zero).  Output: the correction of level T in its e, or, when T
// is level 0, added to phi.
struct TailLevel {
    float *e, *f, *r, *ap, *am, *b, *d;
    int nz, nr;
};

__device__ __forceinline__ void tail_half_sweep(const TailLevel& L, int color) {
    const int W = L.nr + 1;
    const int n = (L.nz - 1) * W;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int i = 1 + q / W, j = q - (i - 1) * W;
        if (((i + j) & 1) != color) continue;
        const int k = i * W + j;
        float v = L.f[k];
        if (j < L.nr) v += L.ap[j] * L.e[k + 1];
        if (j > 0) v += L.am[j] * L.e[k - 1];
        if (i + 1 < L.nz) v += L.b[j] * L.e[k + W];
        if (i - 1 > 0) v += L.b[j] * L.e[k - W];
        L.e[k] = v * L.d[j];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(TAIL_THREADS) k_mg_tail(const MGLevel* lev, const MGTop* top, const int* nlev,
                                                          const int* tail_lev, const int* done,
                                                          const float* const* inv, int sweeps) {
    extern __shared__ float sm[];
    __shared__ TailLevel tl[MG_MAX_LEVELS];
    const int run = blockIdx.x;
    if (done[run]) return;
    const int n = nlev[run], T = tail_lev[run];
    const MGLevel* Lg = lev + run * MG_MAX_LEVELS;
    if (threadIdx.x == 0) {
        int o = 0;
        for (int l = T; l < n; ++l) {
            const int W = Lg[l].nr + 1, nodes = (Lg[l].nz + 1) * W;
            TailLevel& t = tl[l];
            t.nz = Lg[l].nz;
            t.nr = Lg[l].nr;
            t.e = sm + o;
            t.f = t.e + nodes;
            t.r = t.f + nodes;
            t.ap = t.r + nodes;
            t.am = t.ap + W;
            t.b = t.am + W;
            t.d = t.b + W;
            o += 3 * nodes + 4 * W;
        }
    }
    __syncthreads();
    // inputs: f of level T, zero corrections, the coefficients
    for (int l = T; l < n; ++l) {
        const TailLevel t = tl[l];
        const int W = t.nr + 1, nodes = (t.nz + 1) * W;
        for (int k = threadIdx.x; k < nodes; k += blockDim.x) {
            t.e[k] = 0.0f;
            if (l == T) t.f[k] = Lg[l].f[k];
        }
        for (int j = threadIdx.x; j < W; j += blockDim.x) {
            t.ap[j] = Lg[l].ap[j];
            t.am[j] = Lg[l].am[j];
            t.b[j] = Lg[l].b[j];
            t.d[j] = Lg[l].dinv[j];
        }
    }
    __syncthreads();
    // down
    for (int l = T; l + 1 < n; ++l) {
        const TailLevel F = tl[l], Cl = tl[l + 1];
        for (int k = 0; k < 4; ++k) tail_half_sweep(F, k & 1);
        const int Wf = F.nr + 1, Wc = Cl.nr + 1;
        for (int q = threadIdx.x; q < (F.nz - 1) * Wf; q += blockDim.x) {
            const int i = 1 + q / Wf, j = q - (i - 1) * Wf;
            const int k = i * Wf + j;
            float s = (F.ap[j] + F.am[j] + 2.0f * F.b[j]) * F.e[k];
            if (j < F.nr) s -= F.ap[j] * F.e[k + 1];
            if (j > 0) s -= F.am[j] * F.e[k - 1];
            if (i + 1 < F.nz) s -= F.b[j] * F.e[k + Wf];
            if (i - 1 > 0) s -= F.b[j] * F.e[k - Wf];
            F.r[k] = F.f[k] - s;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < (Cl.nz + 1) * Wc; k += blockDim.x) {
            const int I = k / Wc, J = k - I * Wc;
            if (I == 0 || I == Cl.nz) {
                Cl.f[k] = 0.0f;
                continue;
            }
            float s = 0.0f;
            for (int di = -1; di <= 1; ++di) {
                const int i = 2 * I + di;
                if (i <= 0 || i >= F.nz) continue;
                const float wi = di == 0 ? 1.0f : 0.5f;
                for (int dj = -1; dj <= 1; ++dj) {
                    const int j = 2 * J + dj;
                    if (j < 0 || j > F.nr) continue;
                    const float wj = dj == 0 ? 1.0f : 0.5f;
                    s += wi * wj * F.r[i * Wf + j];
                }
            }
            Cl.f[k] = s;
        }
        __syncthreads();
    }
    // coarsest
    {
        const TailLevel L = tl[n - 1];
        const int W = L.nr + 1;
        const int m = (L.nz - 1) * W;
        const float* Ai = inv[run];
        if (Ai) {
            // e = A^-1 f: P threads per unknown, each summing every P-th
            // term (their loads in flight together), then a shuffle sum
            const int P = m <= 64 ? 8 : (m <= 128 ? 4 : (m <= 256 ? 2 : 1));
            const int per = (int)blockDim.x / P;
            for (int u0 = 0; u0 < m; u0 += per) {        // the same trip count in every thread
                const int u = u0 + (int)threadIdx.x / P, part = (int)threadIdx.x % P;
                float acc = 0.0f;
                if (u < m) {
#pragma unroll 8
                    for (int v = part; v < m; v += P) acc += Ai[(size_t)v * m + u] * L.f[W + v];
                }
                for (int o = P >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o, P);
                if (part == 0 && u < m) L.e[W + u] = acc;
            }
            __syncthreads();
        } else {
            for (int it = 0; it < sweeps; ++it) {
                tail_half_sweep(L, 0);
                tail_half_sweep(L, 1);
            }
        }
    }
    // up
    for (int l = n - 2; l >= T; --l) {
        const TailLevel F = tl[l], Cl = tl[l + 1];
        const int Wf = F.nr + 1, Wc = Cl.nr + 1;
        for (int q = threadIdx.x; q < (F.nz - 1) * Wf; q += blockDim.x) {
            const int i = 1 + q / Wf, j = q - (i - 1) * Wf;
            const int I0 = i >> 1, J0 = j >> 1;
            const int I1 = (i & 1) ? I0 + 1 : I0, J1 = (j & 1) ? J0 + 1 : J0;
            const float c = 0.25f * (Cl.e[I0 * Wc + J0] + Cl.e[I1 * Wc + J0] + Cl.e[I0 * Wc + J1] + Cl.e[I1 * Wc + J1]);
            F.e[i * Wf + j] += c;
        }
        __syncthreads();
        for (int k = 0; k < 4; ++k) tail_half_sweep(F, 1 - (k & 1));
    }
    // output
    const TailLevel t = tl[T];
    const int W = t.nr + 1;
    if (T == 0) {
        double* phi = top[run].phi;
        for (int q = threadIdx.x; q < (t.nz - 1) * W; q += blockDim.x) phi[W + q] += (double)t.e[W + q];
    } else {
        float* e = Lg[T].e;
        for (int k = threadIdx.x; k < (t.nz + 1) * W; k += blockDim.x) e[k] = t.e[k];
    }
}

// E = -grad(phi): central inside, one-sided at the electrodes, E_r = 0 on the
// axis and at r = R
__global__ void k_efield(const MGTop* top, const RunInfo* runs, float2* E) {
    const int run = blockIdx.y;
    const MGTop T = top[run];
    const int nz = T.nz, nr = T.nr;
    const int W = nr + 1;
    const int n = (nz + 1) * W;
    const double* p = T.phi;
    float2* out = E + runs[run].node_base;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = k / W, j = k - i * W;
        double ez, er;
        if (i == 0) ez = -(p[k + W] - p[k]) * T.idz;
        else if (i == nz) ez = -(p[k] - p[k - W]) * T.idz;
        else ez = -(p[k + W] - p[k - W]) * T.i2dz;
        if (j == 0 || j == nr) er = 0.0;
        else er = -(p[k + 1] - p[k - 1]) * T.i2dr;
        out[k] = make_float2((float)ez, (float)er);
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

// coefficients of one level (cell sizes dz, dr, nr cells radially)
static void level_coeffs(int nr, double dz, double dr, std::vector<double>& ap, std::vector<double>& am,
                         std::vector<double>& bb) {
    ap.assign(nr + 1, 0.0);
    am.assign(nr + 1, 0.0);
    bb.assign(nr + 1, 0.0);
    const double Rr = nr * dr;
    for (int j = 0; j <= nr; ++j) {
        const double rp = (j + 0.5) * dr, rm = (j - 0.5) * dr;
        ap[j] = j < nr ? 2.0 * PI_ * rp * dz / dr : 0.0;
        am[j] = j > 0 ? 2.0 * PI_ * rm * dz / dr : 0.0;
        double A;
        if (j == 0) A = PI_ * (0.5 * dr) * (0.5 * dr);
        else if (j == nr) A = PI_ * (Rr * Rr - (Rr - 0.5 * dr) * (Rr - 0.5 * dr));
        else A = 2.0 * PI_ * j * dr * dr;
        bb[j] = A / dz;
    }
}

template <typename T>
static void upload(T* dst, const std::vector<T>& v, cudaStream_t s) {
    cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

static std::vector<float> to_float(const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); }

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
    // every array starts at zero (the electrode rows of the corrections stay zero)
    if (cudaMemsetAsync(ws, 0, bytes, s) != cudaSuccess) return 1;
    fs.nruns = R;
    fs.nlev.assign(R, 0);
    fs.host_lev.assign((size_t)R * MG_MAX_LEVELS, MGLevel{});
    fs.host_top.assign(R, MGTop{});
    fs.max_levels = 0;
    fs.max_tail = 0;
    fs.tail_smem = 0;
    fs.tail_lev.assign(R, 0);
    fs.max_nodes0 = 0;
    fs.max_cycles = cfgs[0].poisson_max_cycles > 0 ? cfgs[0].poisson_max_cycles : 60;
    std::vector<double> tol(R);
    std::vector<float*> inv(R, nullptr);
    for (int r = 0; r < R; ++r) {
        const pd_config& c = cfgs[r];
        int a[MG_MAX_LEVELS], b[MG_MAX_LEVELS], n;
        level_dims(c.nz, c.nr, a, b, n);
        fs.nlev[r] = n;
        fs.max_levels = std::max(fs.max_levels, n);
        fs.tail_lev[r] = tail_level(a, b, n);
        fs.max_tail = std::max(fs.max_tail, fs.tail_lev[r]);
        fs.tail_smem = std::max(fs.tail_smem, tail_floats(a, b, n) * sizeof(float));
        fs.max_nodes0 = std::max(fs.max_nodes0, (c.nz + 1) * (c.nr + 1));
        tol[r] = c.poisson_tol;
        // level 0 in double
        MGTop& T = fs.host_top[r];
        const size_t W0 = (size_t)c.nr + 1, nodes0 = ((size_t)c.nz + 1) * W0;
        T.nz = c.nz;
        T.nr = c.nr;
        T.phi = phi + node_base[r];
        T.bf = (double*)take(nodes0 * 8);
        T.ap = (double*)take(W0 * 8);
        T.am = (double*)take(W0 * 8);
        T.b = (double*)take(W0 * 8);
        T.dg = (double*)take(W0 * 8);
        T.cr = (double*)take(W0 * 8);
        T.iv = (double*)take(W0 * 8);
        T.idz = 1.0 / c.dz;
        T.i2dz = 1.0 / (2.0 * c.dz);
        T.i2dr = 1.0 / (2.0 * c.dr);
        std::vector<double> ap, am, bb;
        level_coeffs(c.nr, c.dz, c.dr, ap, am, bb);
        std::vector<double> cr(W0), iv(W0);
        const double qw = QE_ * c.weight / 4294967296.0;
        for (int j = 0; j <= c.nr; ++j) {
            double verb;     // Verboncoeur volume of an interior node
            if (j == 0) verb = PI_ * c.dz * c.dr * c.dr / 3.0;
            else if (j == c.nr) verb = 2.0 * PI_ * c.dz * c.dr * c.dr * ((double)c.nr / 2.0 - 1.0 / 6.0);
            else verb = 2.0 * PI_ * c.dz * c.dr * c.dr * (double)j;
            const double vfv = bb[j] * c.dz * c.dz;   // finite volume: radial extent area x dz
            iv[j] = 1.0 / verb;
            cr[j] = qw * vfv / (verb * EPS0_);        // b = (charge / verb) vfv / eps0
        }
        upload(T.ap, ap, s);
        upload(T.am, am, s);
        upload(T.b, bb, s);
        std::vector<double> dg(W0);
        for (size_t j = 0; j < W0; ++j) dg[j] = ap[j] + am[j] + 2.0 * bb[j];
        upload(T.dg, dg, s);
        upload(T.cr, cr, s);
        upload(T.iv, iv, s);
        cudaStreamSynchronize(s);          // the host vectors above go out of scope
        // correction levels in float
        for (int l = 0; l < n; ++l) {
            MGLevel& L = fs.host_lev[(size_t)r * MG_MAX_LEVELS + l];
            L.nz = a[l];
            L.nr = b[l];
            const double dz = c.dz * (double)(1 << l), dr = c.dr * (double)(1 << l);
            const size_t W = (size_t)L.nr + 1, nodes = ((size_t)L.nz + 1) * W;
            L.e = (float*)take(nodes * 4);
            L.e2 = (float*)take(nodes * 4);
            L.f = (float*)take(nodes * 4);
            L.ap = (float*)take(W * 4);
            L.am = (float*)take(W * 4);
            L.b = (float*)take(W * 4);
            L.dinv = (float*)take(W * 4);
            std::vector<double> lap, lam, lbb;
            level_coeffs(L.nr, dz, dr, lap, lam, lbb);
            std::vector<double> dinv(W);
            for (size_t j = 0; j < W; ++j) dinv[j] = 1.0 / (lap[j] + lam[j] + 2.0 * lbb[j]);
            const std::vector<float> fap = to_float(lap), fam = to_float(lam), fbb = to_float(lbb),
                                     fdi = to_float(dinv);
            upload(L.ap, fap, s);
            upload(L.am, fam, s);
            upload(L.b, fbb, s);
            upload(L.dinv, fdi, s);
            std::vector<float> fai;
            if (l == n - 1 && coarse_unknowns(a, b, n) <= MG_DIRECT_MAX) {
                const int m = coarse_unknowns(a, b, n);
                std::vector<double> Ai;
                if (!invert_coarse(L.nz, L.nr, lap, lam, lbb, Ai)) return 1;
                inv[r] = (float*)take((size_t)m * m * 4);
                fai = to_float(Ai);
                upload(inv[r], fai, s);
            }
            cudaStreamSynchronize(s);      // the host vectors above go out of scope
        }
    }
    fs.lev = (MGLevel*)take((size_t)R * MG_MAX_LEVELS * sizeof(MGLevel));
    fs.top = (MGTop*)take((size_t)R * sizeof(MGTop));
    fs.nlev_dev = (int*)take((size_t)R * 4);
    fs.tail_lev_dev = (int*)take((size_t)R * 4);
    fs.done = (int*)take((size_t)R * 4);
    fs.red = (double*)take((size_t)R * RED_BLOCKS * 2 * 8);
    fs.bnorm = (double*)take((size_t)R * 8);
    fs.tol = (double*)take((size_t)R * 8);
    fs.inv = (float**)take((size_t)R * sizeof(float*));
    // work lists, level by level: the levels above each run's tail
    std::vector<int2> tasks;
    for (int l = 0; l < MG_MAX_LEVELS; ++l) {
        auto add = [&](int r, long long cnt, int step) {
            for (long long q = 0; q < cnt; q += step) tasks.push_back(make_int2(r, (int)q));
        };
        fs.coarse_off[l] = (int)tasks.size();
        for (int r = 0; r < R; ++r)
            if (l < fs.tail_lev[r]) {
                const MGLevel& C = fs.host_lev[(size_t)r * MG_MAX_LEVELS + l + 1];
                add(r, (long long)(C.nz + 1) * (C.nr + 1), MAP_CHUNK);
            }
        fs.coarse_len[l] = (int)tasks.size() - fs.coarse_off[l];
        fs.tile_off[l] = (int)tasks.size();
        for (int r = 0; r < R; ++r)
            if (l < fs.tail_lev[r]) {
                const MGLevel& L = fs.host_lev[(size_t)r * MG_MAX_LEVELS + l];
                add(r, tiles_of(L.nz, L.nr), 1);
            }
        fs.tile_len[l] = (int)tasks.size() - fs.tile_off[l];
    }
    if (fs.tail_smem > 48 * 1024) return 1;          // cannot happen: tail levels hold at most 34 x 34 nodes
    fs.tasks = (int2*)take(tasks.size() * sizeof(int2) + 8);
    if (o > bytes) return 1;
    upload(fs.tasks, tasks, s);
    upload(fs.lev, fs.host_lev, s);
    upload(fs.top, fs.host_top, s);
    upload(fs.nlev_dev, fs.nlev, s);
    upload(fs.tail_lev_dev, fs.tail_lev, s);
    upload(fs.tol, tol, s);
    upload(fs.inv, inv, s);
    if (!fs.host_done && cudaMallocHost(&fs.host_done, (size_t)R * 4) != cudaSuccess) return 1;
    return cudaStreamSynchronize(s) == cudaSuccess ? 0 : 1;
}

void field_free(FieldSolver& fs) {
    if (fs.host_done) cudaFreeHost(fs.host_done);
    fs.host_done = nullptr;
}

// two red-black iterations (four half-sweeps) in one launch: pre-smoothing
// from zero into e2, or post-smoothing from e2 plus the prolongated
// correction of level l + 1 into e (level 0: into phi)
static int smooth4(FieldSolver& fs, int l, bool post, cudaStream_t s) {
    if (!fs.tile_len[l]) return 0;
    const int2* t = fs.tasks + fs.tile_off[l];
    if (!post) k_smooth4<false, false><<<fs.tile_len[l], 256, 0, s>>>(fs.lev, fs.top, fs.done, l, t);
    else if (l == 0) k_smooth4<true, true><<<fs.tile_len[l], 256, 0, s>>>(fs.lev, fs.top, fs.done, l, t);
    else k_smooth4<true, false><<<fs.tile_len[l], 256, 0, s>>>(fs.lev, fs.top, fs.done, l, t);
    return 1;
}

// one correction cycle of every run that has not converged (the right-hand
// side is level 0's f, set with the residual norms); returns the kernels
// launched
static int vcycle(FieldSolver& fs, cudaStream_t s) {
    const int R = fs.nruns;
    const int th = fs.threads;
    int nk = 0;
    // down to each run's tail: pre-smooth, residual and restriction
    for (int l = 0; l < fs.max_tail; ++l) {
        nk += smooth4(fs, l, false, s);
        if (fs.coarse_len[l]) {
            k_restrict<<<fs.coarse_len[l], th, 0, s>>>(fs.lev, fs.done, l, fs.tasks + fs.coarse_off[l]);
            ++nk;
        }
    }
    // the tail levels of every run, one block each
    k_mg_tail<<<R, TAIL_THREADS, fs.tail_smem, s>>>(fs.lev, fs.top, fs.nlev_dev, fs.tail_lev_dev, fs.done, fs.inv,
                                                    200);
    ++nk;
    // up: prolongation and post-smoothing in one launch per level; level 0's adds the correction to phi
    for (int l = fs.max_tail - 1; l >= 0; --l) nk += smooth4(fs, l, true, s);
    return nk;
}

static void norms(FieldSolver& fs, RunState* rs, int cycle, int first, cudaStream_t s) {
    const int R = fs.nruns;
    const dim3 g(RED_BLOCKS, R);
    k_residual_norms<<<g, 256, 0, s>>>(fs.top, fs.lev, fs.nlev_dev, fs.red, first);
    k_norms<<<(R + 3) / 4, 128, 0, s>>>(fs.red, fs.bnorm, fs.done, fs.tol, rs, R, cycle, first);
}

cudaError_t field_solve(FieldSolver& fs, const long long* rho_e, const long long* rho_h, double* phi, float2* E,
                const RunInfo* runs, RunState* rs, int host_check, int cycles, cudaStream_t s, int* kernels) {
    (void)E;
    (void)phi;
    const int R = fs.nruns;
    const dim3 g0(blocks_for(fs, fs.max_nodes0), R);
    k_rhs<<<g0, fs.threads, 0, s>>>(rho_e, rho_h, fs.top, runs, rs);
    norms(fs, rs, 0, 1, s);
    if (kernels) *kernels += 3;
    if (host_check) {
        for (int cyc = 1; cyc <= fs.max_cycles; ++cyc) {
            cudaError_t e = cudaMemcpyAsync(fs.host_done, fs.done, (size_t)R * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
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
    return cudaGetLastError();
}

// E for every run (separate so the caller can time it)
void field_efield(FieldSolver& fs, const double* phi, const RunInfo* runs, float2* E, DevState* st, RunState* rs,
                  cudaStream_t s) {
    (void)phi;
    const dim3 g(blocks_for(fs, fs.max_nodes0), fs.nruns);
    k_efield<<<g, fs.threads, 0, s>>>(fs.top, runs, E);
    k_solve_epilogue<<<1, 128, 0, s>>>(fs.done, fs.nruns, st, rs);
}

// ------------------------------------------------------------------
// warm start
// ------------------------------------------------------------------
// node density of the current fixed-point charge (C/m^3)
__device__ __forceinline__ double node_rho(const long long* rho_e, const long long* rho_h, const MGTop& T,
                                           double qw, int i, int j, uint32_t g) {
    const double f = (i == 0 || i == T.nz) ? 2.0 : 1.0;       // half volume on the electrode rows
    return qw * (double)(rho_e[g] + rho_h[g]) * (T.iv[j] * f);
}

// history shift at the start of a solve: rho_prev2 := rho_prev, rho_prev :=
// rho_last, phi_prev2 := phi_prev, phi_prev := phi, V_prev2 := V_prev,
// V_prev := V_last; then rho_last := current density, V_last := V
__global__ void k_warm_history(const long long* rho_e, const long long* rho_h, const MGTop* top,
                               const RunInfo* runs, const RunState* rs, WarmHistory h, int extrapolate) {
    const int run = blockIdx.y;
    const MGTop T = top[run];
    const RunInfo& RI = runs[run];
    const double qw = QE_ * RI.weight / 4294967296.0;
    const int W = T.nr + 1, n = (T.nz + 1) * W;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = k / W, j = k - i * W;
        const uint32_t g = RI.node_base + (uint32_t)k;
        h.rho_prev2[g] = h.rho_prev[g];
        h.rho_prev[g] = h.rho_last[g];
        const double p = T.phi[k], pp = h.phi_prev[g];
        if (extrapolate && i > 0 && i < T.nz) T.phi[k] = 2.0 * p - pp;
        h.phi_prev2[g] = pp;
        h.phi_prev[g] = p;
        h.rho_last[g] = node_rho(rho_e, rho_h, T, qw, i, j, g);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        h.V_prev2[run] = h.V_prev[run];
        h.V_prev[run] = h.V_last[run];
        h.V_last[run] = rs[run].V;
    }
}

// The references of a form: d = rho_last - c1 rho1 - c2 rho2 and base =
// c1 phi1 + c2 phi2 + (V - c1 V1 - c2 V2) z / L (absent terms: 0)
struct WarmRef {
    const double *rho1, *rho2, *phi1, *phi2, *V1, *V2;
    double c1, c2;
};

WarmRef warm_ref(const WarmHistory& h, int form) {
    WarmRef r{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, 0.0};
    if (form == WARM_DELTA) {
        r.rho1 = h.rho_prev;
        r.phi1 = h.phi_prev;
        r.V1 = h.V_prev;
        r.c1 = 1.0;
    } else if (form == WARM_EXTRAP) {
        r.rho1 = h.rho_prev;
        r.phi1 = h.phi_prev;
        r.V1 = h.V_prev;
        r.c1 = 2.0;
        r.rho2 = h.rho_prev2;
        r.phi2 = h.phi_prev2;
        r.V2 = h.V_prev2;
        r.c2 = -1.0;
    }
    return r;
}

__device__ __forceinline__ double warm_d(const double* rho_last, const WarmRef& R, uint32_t g) {
    double d = rho_last[g];
    if (R.rho1) d -= R.c1 * R.rho1[g];
    if (R.rho2) d -= R.c2 * R.rho2[g];
    return d;
}

// rmax[run] = max |d|
__global__ void k_warm_rmax(const double* rho_last, WarmRef R, const RunInfo* runs, unsigned long long* rmax_bits) {
    const int run = blockIdx.y;
    const RunInfo& RI = runs[run];
    const int n = (RI.nz + 1) * (RI.nr + 1);
    double m = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        m = fmax(m, fabs(warm_d(rho_last, R, RI.node_base + (uint32_t)k)));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xFFFFFFFFu, m, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(&rmax_bits[run], (unsigned long long)__double_as_longlong(m));
}

__global__ void k_warm_x(const double* rho_last, WarmRef R, const RunInfo* runs, const double* rmax, float* x) {
    const int run = blockIdx.y;
    const RunInfo& RI = runs[run];
    const int n = (RI.nz + 1) * (RI.nr + 1);
    const double rm = rmax[run];
    const double irm = rm > 0.0 ? 1.0 / rm : 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t g = RI.node_base + (uint32_t)k;
        x[g] = (float)(warm_d(rho_last, R, g) * irm);
    }
}

// the potential the prediction is added to
__device__ __forceinline__ double warm_base(const WarmRef& R, int run, double V, uint32_t g, int i, double inz) {
    double b = 0.0, Vr = 0.0;
    if (R.phi1) {
        b += R.c1 * R.phi1[g];
        Vr += R.c1 * R.V1[run];
    }
    if (R.phi2) {
        b += R.c2 * R.phi2[g];
        Vr += R.c2 * R.V2[run];
    }
    return b + (V - Vr) * ((double)i * inz);
}

__global__ void k_warm_apply(const float* y, const MGTop* top, const RunInfo* runs, const RunState* rs,
                             const double* rmax, WarmRef R, double* phi) {
    const int run = blockIdx.y;
    const RunInfo& RI = runs[run];
    const MGTop T = top[run];
    const int W = RI.nr + 1, n = (RI.nz - 1) * W;
    const double V = rs[run].V, inz = 1.0 / (double)RI.nz;
    const double dz = 1.0 / T.idz;
    const double sc = y ? rmax[run] * dz * dz / EPS0_ : 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int i = 1 + q / W;
        const uint32_t g = RI.node_base + (uint32_t)(W + q);
        const double base = warm_base(R, run, V, g, i, inz);
        phi[g] = y ? base + (double)y[g] * sc : base;
    }
}

__global__ void k_warm_targets(const double* phi, const MGTop* top, const RunInfo* runs, const double* V_last,
                               const double* rmax, WarmRef R, float* t) {
    const int run = blockIdx.y;
    const RunInfo& RI = runs[run];
    const MGTop T = top[run];
    const int W = RI.nr + 1, n = (RI.nz + 1) * W;
    const double V = V_last[run], rm = rmax[run], inz = 1.0 / (double)RI.nz;
    const double dz = 1.0 / T.idz;
    const double sc = rm > 0.0 ? EPS0_ / (rm * dz * dz) : 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = k / W;
        const uint32_t g = RI.node_base + (uint32_t)k;
        t[g] = (float)((phi[g] - warm_base(R, run, V, g, i, inz)) * sc);
    }
}

void warm_history(FieldSolver& fs, const long long* rho_e, const long long* rho_h, const RunInfo* runs,
                  const RunState* rs, double* phi, const WarmHistory& h, bool extrapolate, cudaStream_t s) {
    (void)phi;
    const dim3 g(blocks_for(fs, fs.max_nodes0), fs.nruns);
    k_warm_history<<<g, fs.threads, 0, s>>>(rho_e, rho_h, fs.top, runs, rs, h, extrapolate ? 1 : 0);
}

void warm_inputs(FieldSolver& fs, const WarmHistory& h, int form, const RunInfo* runs, double* rmax, float* x,
                 cudaStream_t s) {
    const dim3 g(blocks_for(fs, fs.max_nodes0), fs.nruns);
    const WarmRef R = warm_ref(h, form);
    cudaMemsetAsync(rmax, 0, (size_t)fs.nruns * 8, s);
    k_warm_rmax<<<g, fs.threads, 0, s>>>(h.rho_last, R, runs, (unsigned long long*)rmax);
    k_warm_x<<<g, fs.threads, 0, s>>>(h.rho_last, R, runs, rmax, x);
}

void warm_apply(FieldSolver& fs, const float* y, const WarmHistory& h, int form, const RunInfo* runs,
                const RunState* rs, const double* rmax, double* phi, cudaStream_t s) {
    const dim3 g(blocks_for(fs, fs.max_nodes0), fs.nruns);
    k_warm_apply<<<g, fs.threads, 0, s>>>(y, fs.top, runs, rs, rmax, warm_ref(h, form), phi);
}

void warm_targets(FieldSolver& fs, const double* phi, const WarmHistory& h, int form, const RunInfo* runs,
                  const double* rmax, float* t, cudaStream_t s) {
    const dim3 g(blocks_for(fs, fs.max_nodes0), fs.nruns);
    k_warm_targets<<<g, fs.threads, 0, s>>>(phi, fs.top, runs, h.V_last, rmax, warm_ref(h, form), t);
}

}  // namespace pd
