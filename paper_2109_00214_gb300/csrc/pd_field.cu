// pd_field.cu -- Poisson solve of Eq. (8), read as lap(phi) = -rho/eps0, by
// geometric multigrid on the r-z node grid, and E = -grad(phi).
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
// bilinear prolongation, coefficients rediscretised on each level, and a
// single-block Gauss-Seidel solve on the coarsest level.  Double precision;
// the cycle stops once |b - A phi| / |b| <= tol (checked on the host between
// cycles).
#include <cmath>
#include <cstring>
#include <vector>

#include "pd_field.h"

namespace pd {

namespace {
constexpr double QE_ = 1.602176634e-19;
constexpr double EPS0_ = 8.8541878128e-12;
constexpr double PI_ = 3.14159265358979323846;

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

void level_dims(int nz, int nr, int* nzs, int* nrs, int& nlev) {
    nlev = 0;
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
}  // namespace

bool field_grid_ok(int nz, int nr) {
    int a[MG_MAX_LEVELS], b[MG_MAX_LEVELS], n;
    level_dims(nz, nr, a, b, n);
    return (a[n - 1] + 1) * (b[n - 1] + 1) <= 1024 && a[n - 1] >= 2 && b[n - 1] >= 2;
}

size_t field_workspace_bytes(int nz, int nr) {
    int a[MG_MAX_LEVELS], b[MG_MAX_LEVELS], n;
    level_dims(nz, nr, a, b, n);
    size_t t = 0;
    for (int l = 0; l < n; ++l) {
        const size_t nodes = (size_t)(a[l] + 1) * (b[l] + 1);
        t += 3 * al(nodes * 8) + 3 * al((size_t)(b[l] + 1) * 8);
    }
    t += 2 * al((size_t)(nr + 1) * 8) + al(4096 * 8);
    return t;
}

// ------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------
__global__ void k_rhs(const long long* rho_e, const long long* rho_h, const double* fv_over_verb,
                      const double* verb_base, MGLevel L, double qw, const DevState* st, double* phi) {
    const int W = L.nr + 1;
    const int n = (L.nz + 1) * W;
    const double V = st->V;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = k / W, j = k - i * W;
        if (i == 0) {
            phi[k] = 0.0;
            L.f[k] = 0.0;
            continue;
        }
        if (i == L.nz) {
            phi[k] = V;
            L.f[k] = 0.0;
            continue;
        }
        // rho_ij (C/m^3) = q W rho_int 2^-32 / V_verb; rhs = rho Vfv / eps0
        const double rho = qw * (double)(rho_e[k] + rho_h[k]) / verb_base[j];
        double v = rho * (fv_over_verb[j] * verb_base[j]) / EPS0_;
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

// red-black Gauss-Seidel on the interior rows; Dirichlet neighbours are part
// of f (level 0) or zero (corrections)
__global__ void k_smooth(MGLevel L, int color) {
    const int W = L.nr + 1;
    const int n = (L.nz - 1) * W;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
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
}

__global__ void k_residual(MGLevel L, double* red) {
    const int W = L.nr + 1;
    const int n = (L.nz - 1) * W;
    double acc = 0.0, accb = 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int i = 1 + q / W, j = q - (i - 1) * W;
        const int k = i * W + j;
        const double r = L.f[k] - apply_A(L, L.x, i, j);
        L.r[k] = r;
        acc += r * r;
        accb += L.f[k] * L.f[k];
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
            red[2 * blockIdx.x] = t;
            red[2 * blockIdx.x + 1] = tb;
        }
    }
}

// coarse rhs = sum of the fine integrated residuals over the coarse control
// volume (full weighting scaled by 4); zero initial coarse correction
__global__ void k_restrict(MGLevel F, MGLevel Cl) {
    const int Wc = Cl.nr + 1, Wf = F.nr + 1;
    const int n = (Cl.nz + 1) * Wc;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
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

__global__ void k_prolong(MGLevel F, MGLevel Cl) {
    const int Wc = Cl.nr + 1, Wf = F.nr + 1;
    const int n = (F.nz - 1) * Wf;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int i = 1 + q / Wf, j = q - (i - 1) * Wf;
        const int I0 = i >> 1, J0 = j >> 1;
        const int I1 = (i & 1) ? I0 + 1 : I0, J1 = (j & 1) ? J0 + 1 : J0;
        const double c = 0.25 * (Cl.x[I0 * Wc + J0] + Cl.x[I1 * Wc + J0] + Cl.x[I0 * Wc + J1] + Cl.x[I1 * Wc + J1]);
        F.x[i * Wf + j] += c;
    }
}

// coarsest level: Gauss-Seidel sweeps in one block
__global__ void __launch_bounds__(1024) k_coarse(MGLevel L, int sweeps) {
    const int W = L.nr + 1;
    const int n = (L.nz - 1) * W;
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
__global__ void k_efield(const double* phi, int nz, int nr, double dz, double dr, float2* E) {
    const int W = nr + 1;
    const int n = (nz + 1) * W;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = k / W, j = k - i * W;
        double ez, er;
        if (i == 0) ez = -(phi[k + W] - phi[k]) / dz;
        else if (i == nz) ez = -(phi[k] - phi[k - W]) / dz;
        else ez = -(phi[k + W] - phi[k - W]) / (2.0 * dz);
        if (j == 0 || j == nr) er = 0.0;
        else er = -(phi[k + 1] - phi[k - 1]) / (2.0 * dr);
        E[k] = make_float2((float)ez, (float)er);
    }
}

__global__ void k_record(DevState* st, double relres, double cycles, int bad) {
    st->relres = relres;
    st->cycles = cycles;
    if (bad) atomicOr(&st->error, ERR_NONFINITE);
}

// ------------------------------------------------------------------
// host
// ------------------------------------------------------------------
static int blocks_for(int n) {
    int b = (n + 255) / 256;
    return b < 1 ? 1 : (b > 1216 ? 1216 : b);
}

int field_init(FieldSolver& fs, const pd_config& c, void* ws, size_t bytes, cudaStream_t s) {
    int a[MG_MAX_LEVELS], b[MG_MAX_LEVELS], n;
    level_dims(c.nz, c.nr, a, b, n);
    char* w = (char*)ws;
    size_t o = 0;
    auto take = [&](size_t sz) {
        char* p = w + o;
        o += al(sz);
        return p;
    };
    fs.nlev = n;
    fs.nz = c.nz;
    fs.nr = c.nr;
    fs.weight = c.weight;
    fs.tol = c.poisson_tol;
    fs.max_cycles = c.poisson_max_cycles > 0 ? c.poisson_max_cycles : 60;
    fs.V0 = c.V0;
    for (int l = 0; l < n; ++l) {
        MGLevel& L = fs.lev[l];
        L.nz = a[l];
        L.nr = b[l];
        L.dz = c.dz * (double)(1 << l);
        L.dr = c.dr * (double)(1 << l);
        const size_t nodes = (size_t)(L.nz + 1) * (L.nr + 1);
        L.x = (double*)take(nodes * 8);
        L.f = (double*)take(nodes * 8);
        L.r = (double*)take(nodes * 8);
        L.ap = (double*)take((size_t)(L.nr + 1) * 8);
        L.am = (double*)take((size_t)(L.nr + 1) * 8);
        L.b = (double*)take((size_t)(L.nr + 1) * 8);
        std::vector<double> ap(L.nr + 1), am(L.nr + 1), bb(L.nr + 1);
        const double R = L.nr * L.dr;
        for (int j = 0; j <= L.nr; ++j) {
            const double rp = (j + 0.5) * L.dr, rm = (j - 0.5) * L.dr;
            ap[j] = j < L.nr ? 2.0 * PI_ * rp * L.dz / L.dr : 0.0;
            am[j] = j > 0 ? 2.0 * PI_ * rm * L.dz / L.dr : 0.0;
            double A;
            if (j == 0) A = PI_ * (0.5 * L.dr) * (0.5 * L.dr);
            else if (j == L.nr) A = PI_ * (R * R - (R - 0.5 * L.dr) * (R - 0.5 * L.dr));
            else A = 2.0 * PI_ * j * L.dr * L.dr;
            bb[j] = A / L.dz;
        }
        cudaMemcpyAsync(L.ap, ap.data(), ap.size() * 8, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(L.am, am.data(), am.size() * 8, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(L.b, bb.data(), bb.size() * 8, cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(L.x, 0, nodes * 8, s);
        if (l == 0) {
            std::vector<double> fvv(L.nr + 1), vb(L.nr + 1);
            for (int j = 0; j <= L.nr; ++j) {
                const double dz = c.dz, dr = c.dr;
                double verb;
                if (j == 0) verb = PI_ * dz * dr * dr / 3.0;
                else if (j == c.nr) verb = 2.0 * PI_ * dz * dr * dr * ((double)c.nr / 2.0 - 1.0 / 6.0);
                else verb = 2.0 * PI_ * dz * dr * dr * (double)j;
                vb[j] = verb;
                const double A = bb[j] * L.dz;  // radial extent area of the control volume
                fvv[j] = A * L.dz / verb;       // Vfv / Vverb, Vfv = A dz
            }
            fs.fv_over_verb = (double*)take(fvv.size() * 8);
            fs.verb_base = (double*)take(vb.size() * 8);
            cudaMemcpyAsync(fs.fv_over_verb, fvv.data(), fvv.size() * 8, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(fs.verb_base, vb.data(), vb.size() * 8, cudaMemcpyHostToDevice, s);
        }
    }
    fs.red = (double*)take(4096 * 8);
    if (o > bytes) return 1;
    if (!fs.host_red && cudaMallocHost(&fs.host_red, 4096 * 8) != cudaSuccess) return 1;
    return cudaStreamSynchronize(s) == cudaSuccess ? 0 : 1;
}

void field_free(FieldSolver& fs) {
    if (fs.host_red) cudaFreeHost(fs.host_red);
    fs.host_red = nullptr;
}

static void vcycle(FieldSolver& fs, int l, cudaStream_t s) {
    MGLevel& L = fs.lev[l];
    const int n = (L.nz + 1) * (L.nr + 1);
    if (l == fs.nlev - 1) {
        k_coarse<<<1, 1024, 0, s>>>(L, 200);
        return;
    }
    for (int it = 0; it < 2; ++it) {
        k_smooth<<<blocks_for(n / 2), 256, 0, s>>>(L, 0);
        k_smooth<<<blocks_for(n / 2), 256, 0, s>>>(L, 1);
    }
    k_residual<<<blocks_for(n), 256, 0, s>>>(L, nullptr);
    MGLevel& Cl = fs.lev[l + 1];
    k_restrict<<<blocks_for((Cl.nz + 1) * (Cl.nr + 1)), 256, 0, s>>>(L, Cl);
    vcycle(fs, l + 1, s);
    k_prolong<<<blocks_for(n), 256, 0, s>>>(L, Cl);
    for (int it = 0; it < 2; ++it) {
        k_smooth<<<blocks_for(n / 2), 256, 0, s>>>(L, 1);
        k_smooth<<<blocks_for(n / 2), 256, 0, s>>>(L, 0);
    }
}

static int residual_norms(FieldSolver& fs, cudaStream_t s, double* rn, double* bn) {
    MGLevel& L = fs.lev[0];
    const int n = (L.nz + 1) * (L.nr + 1);
    const int nb = blocks_for(n) > 2048 ? 2048 : blocks_for(n);
    k_residual<<<nb, 256, 0, s>>>(L, fs.red);
    if (cudaMemcpyAsync(fs.host_red, fs.red, (size_t)nb * 16, cudaMemcpyDeviceToHost, s) != cudaSuccess) return 1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return 1;
    double a = 0, b = 0;
    for (int q = 0; q < nb; ++q) {
        a += fs.host_red[2 * q];
        b += fs.host_red[2 * q + 1];
    }
    *rn = std::sqrt(a);
    *bn = std::sqrt(b);
    return 0;
}

int field_solve(FieldSolver& fs, const long long* rho_e, const long long* rho_h, double* phi, float2* E, DevState* st,
                cudaStream_t s) {
    MGLevel& L0 = fs.lev[0];
    L0.x = phi;   // solve in place; the previous solution is the initial guess
    const int n = (L0.nz + 1) * (L0.nr + 1);
    const double qw = QE_ * fs.weight / 4294967296.0;
    k_rhs<<<blocks_for(n), 256, 0, s>>>(rho_e, rho_h, fs.fv_over_verb, fs.verb_base, L0, qw, st, phi);
    double rn = 0, bn = 0;
    if (residual_norms(fs, s, &rn, &bn)) return 1;
    int cyc = 0;
    bool bad = !std::isfinite(rn) || !std::isfinite(bn);
    while (!bad && bn > 0 && rn > fs.tol * bn && cyc < fs.max_cycles) {
        vcycle(fs, 0, s);
        ++cyc;
        if (residual_norms(fs, s, &rn, &bn)) return 1;
        bad = !std::isfinite(rn);
    }
    k_efield<<<blocks_for(n), 256, 0, s>>>(phi, L0.nz, L0.nr, L0.dz, L0.dr, E);
    k_record<<<1, 1, 0, s>>>(st, bn > 0 ? rn / bn : 0.0, (double)cyc, bad ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace pd
