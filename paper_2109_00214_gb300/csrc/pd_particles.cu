// pd_particles.cu -- scans, the initial deposit and diagnostics.
//
//   k_scan_*    exclusive prefix sum of u32 (bin offsets, candidate offsets).
//   k_deposit   deposit without moving (initial state).
//   diagnostics species counts, density map, energy histogram.
//
// Compiled with -fmad=false: every float operation is rounded on its own, in
// the order written, so results do not depend on contraction choices.
#include "pd_internal.cuh"
#include "pd_kernels.h"
#include "pd_warp.cuh"

namespace pd {

constexpr unsigned FULL = 0xFFFFFFFFu;


// deposit of every live particle without moving (state before the first step)
__global__ void __launch_bounds__(256) k_deposit(Particles A, long long* rho_e, long long* rho_h, DevState* st,
                                                 KParams P) {
    const unsigned long long n = st->n_slots;
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n;
         i0 += stride) {
        const unsigned long long i = i0 + lane;
        const uint32_t key = i < n ? A.key[i] : DEAD;
        const bool live = key != DEAD;
        const int sp = live ? (int)key_species(key) : 0;
        const uint32_t gcell = live ? key_cell(key) : 0u;
        const RunInfo& RI = P.runs[run_of(P, gcell)];
        int iz = 0, ir = 0;
        float pz = 0.f, pr = 0.f;
        const int zq = live ? charge_of(sp) : 0;
        if (live && zq != 0) {
            const uint32_t lc = gcell - RI.cell_base;
            iz = (int)(lc / (uint32_t)RI.nr);
            ir = (int)(lc - (uint32_t)iz * (uint32_t)RI.nr);
            pz = A.pz[i];
            pr = A.pr[i];
        }
        // group lanes by key, which fixes the run, species and cell
        const uint32_t k = live ? make_key((uint32_t)sp, gcell) : DEAD;
        warp_deposit(rho_e, RI, P.geom, k, iz, ir, pz, pr, zq, live && zq != 0 && sp == SP_E);
        warp_deposit(rho_h, RI, P.geom, k, iz, ir, pz, pr, zq, live && zq != 0 && sp != SP_E);
    }
}

// ---------------------------------------------------------------------
// exclusive scan of u32 (input padded to a multiple of SCAN_TILE with zeros)
// ---------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t w = lane < nw ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    const uint32_t wbase = warp > 0 ? warp_sums[warp - 1] : 0u;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return wbase + x - v;
}

// scan input transform: the value itself, or its population count (a scan
// of bit masks counts set bits)
template <bool POPC>
__device__ __forceinline__ uint4 scan_tf(uint4 v) {
    if (POPC) return make_uint4(__popc(v.x), __popc(v.y), __popc(v.z), __popc(v.w));
    return v;
}

template <bool POPC>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t* __restrict__ in, uint32_t* partial,
                                                              const uint32_t* cond) {
    if (cond && !*cond) return;
    const uint4* p = reinterpret_cast<const uint4*>(in + (size_t)blockIdx.x * SCAN_TILE) + threadIdx.x * 2;
    const uint4 a = scan_tf<POPC>(p[0]), b = scan_tf<POPC>(p[1]);
    uint32_t s = (a.x + a.y + a.z + a.w) + (b.x + b.y + b.z + b.w);
    s = __reduce_add_sync(FULL, s);
    __shared__ uint32_t ws[SCAN_THREADS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = threadIdx.x < SCAN_THREADS / 32 ? ws[threadIdx.x] : 0u;
        t = __reduce_add_sync(FULL, t);
        if (threadIdx.x == 0) partial[blockIdx.x] = t;
    }
}

// single block: exclusive scan of nb block sums in place, total to partial[nb]
__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t* partial, uint32_t nb, const uint32_t* cond) {
    if (cond && !*cond) return;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nb; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? partial[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, &tot);
        if (i < nb) partial[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) partial[nb] = carry;
}

template <bool POPC>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const uint32_t* __restrict__ in,
                                                            const uint32_t* __restrict__ partial, uint32_t* out,
                                                            uint32_t n, uint32_t nb, const uint32_t* cond) {
    if (cond && !*cond) return;
    const size_t base = (size_t)blockIdx.x * SCAN_TILE + threadIdx.x * 8;
    const uint4* p = reinterpret_cast<const uint4*>(in + base);
    const uint4 a = scan_tf<POPC>(p[0]), b = scan_tf<POPC>(p[1]);
    uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
    uint32_t tot;
    uint32_t run = partial[blockIdx.x] + block_exclusive_scan(s, &tot);
    uint32_t o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        o[k] = run;
        run += v[k];
    }
    uint4* q = reinterpret_cast<uint4*>(out + base);
    q[0] = make_uint4(o[0], o[1], o[2], o[3]);
    q[1] = make_uint4(o[4], o[5], o[6], o[7]);
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = partial[nb];
}

// ---------------------------------------------------------------------
// diagnostics
// ---------------------------------------------------------------------
// particle slot i belongs to run `run` (cells [cell_base, cell_base + ncell))
__device__ __forceinline__ bool in_run(uint32_t key, const RunInfo& RI) {
    if (key == DEAD) return false;
    const uint32_t c = key_cell(key);
    return c >= RI.cell_base && c < RI.cell_base + RI.ncell;
}

// live particles per species of a single run, out[species]: each thread
// counts its slots in registers, four groups of four keys loaded before any
// is used (independent loads in flight), then a warp sum and one atomic per
// warp and species
__global__ void __launch_bounds__(256) k_species_count1(Particles A, DevState* st, unsigned long long* out) {
    const unsigned long long n = st->n_slots;
    const unsigned long long nv = (n + 3ull) >> 2;           // the slot arrays are padded to four
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const uint4* key4 = reinterpret_cast<const uint4*>(A.key);
    unsigned int c[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) c[k] = 0u;
    for (unsigned long long v0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; v0 < nv;
         v0 += 4ull * stride) {
        uint4 K[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const unsigned long long v = v0 + (unsigned long long)u * stride;
            K[u] = v < nv ? key4[v] : make_uint4(DEAD, DEAD, DEAD, DEAD);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const unsigned long long j0 = 4ull * (v0 + (unsigned long long)u * stride);
            const uint32_t ks[4] = {K[u].x, K[u].y, K[u].z, K[u].w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool live = j0 + (unsigned long long)q < n && ks[q] != DEAD;
                const uint32_t sp = key_species(ks[q]);
#pragma unroll
                for (int k = 0; k < NSP; ++k) c[k] += (live && sp == (uint32_t)k) ? 1u : 0u;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
        const unsigned int w = __reduce_add_sync(FULL, c[k]);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&out[k], (unsigned long long)w);
    }
}

// live particles per run and species, all runs in one pass: out[run * NSP + species]
// (warp-aggregated shared-memory counters, one flush per block)
__global__ void k_species_count_all(Particles A, DevState* st, KParams P, unsigned long long* out) {
    __shared__ unsigned int cnt[MAX_RUNS_SMEM * NSP];
    for (int q = threadIdx.x; q < P.nruns * NSP; q += blockDim.x) cnt[q] = 0u;
    __syncthreads();
    const unsigned long long n = st->n_slots;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n;
         i0 += stride) {
        const unsigned long long i = i0 + (threadIdx.x & 31);
        const uint32_t key = i < n ? A.key[i] : DEAD;
        const bool live = key != DEAD;
        const uint32_t slot = live ? (uint32_t)run_of(P, key_cell(key)) * NSP + key_species(key) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(FULL, slot);
        if (live && (threadIdx.x & 31) == 31 - __clz((int)peers)) atomicAdd(&cnt[slot], (unsigned)__popc(peers));
    }
    __syncthreads();
    for (int q = threadIdx.x; q < P.nruns * NSP; q += blockDim.x)
        if (cnt[q]) atomicAdd(&out[q], (unsigned long long)cnt[q]);
}

__global__ void k_density(Particles A, DevState* st, KParams P, int run, int species, long long* acc) {
    const unsigned long long n = st->n_slots;
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const RunInfo RI = P.runs[run];
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n;
         i0 += stride) {
        const unsigned long long i = i0 + lane;
        const uint32_t key = i < n ? A.key[i] : DEAD;
        const bool on = in_run(key, RI) && (int)key_species(key) == species;
        int iz = 0, ir = 0;
        float pz = 0.f, pr = 0.f;
        if (on) {
            const uint32_t lc = key_cell(key) - RI.cell_base;
            iz = (int)(lc / (uint32_t)RI.nr);
            ir = (int)(lc - (uint32_t)iz * (uint32_t)RI.nr);
            pz = A.pz[i];
            pr = A.pr[i];
        }
        warp_deposit(acc, RI, P.geom, on ? make_key((uint32_t)species, key_cell(key)) : DEAD, iz, ir, pz, pr, 1, on);
    }
}

__global__ void k_spectrum(Particles A, DevState* st, KParams P, int run, int species, double lo, double hi,
                           int nbins, unsigned long long* hist) {
    const unsigned long long n = st->n_slots;
    const double m = P.masses[species];
    const RunInfo RI = P.runs[run];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t key = A.key[i];
        if (!in_run(key, RI) || (int)key_species(key) != species) continue;
        const double vz = A.vz[i], vr = A.vr[i], vt = A.vt[i];
        const double v2 = vz * vz + vr * vr + vt * vt;
        const double e = 0.5 * m * v2 / 1.602176634e-19;
        if (e < lo || e >= hi) continue;
        int b = (int)((e - lo) / (hi - lo) * nbins);
        if (b >= nbins) b = nbins - 1;
        atomicAdd(&hist[b], 1ull);
    }
}

__global__ void k_pack_keys(const uint8_t* __restrict__ sp, const int32_t* __restrict__ iz,
                            const int32_t* __restrict__ ir, const float* __restrict__ pz,
                            const float* __restrict__ pr, long long n, int nz, int nr, uint32_t cell_base, uint32_t id0,
                            uint32_t sp_max, uint32_t* key, uint32_t* id, unsigned int* bad) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int a = iz[q], b = ir[q];
        const uint32_t s = sp[q];
        const float fz = pz[q], fr = pr[q];
        const bool ok = s <= sp_max && a >= 0 && a < nz && b >= 0 && b < nr && fz >= 0.0f && fz < 1.0f && fr >= 0.0f &&
                        fr < 1.0f;
        if (!ok) atomicOr(bad, 1u);
        key[q] = ok ? make_key(s, cell_base + (uint32_t)a * (uint32_t)nr + (uint32_t)b) : DEAD;
        id[q] = id0 + (uint32_t)q;
    }
}

// ---------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------
void launch_deposit(const Particles& A, long long* rho_e, long long* rho_h, DevState* st, const KParams& P,
                    int grid, cudaStream_t s) {
    k_deposit<<<grid, 256, 0, s>>>(A, rho_e, rho_h, st, P);
}
void launch_scan(const uint32_t* in, uint32_t* out, uint32_t* partial, uint32_t n_padded, cudaStream_t s,
                 const uint32_t* cond) {
    const uint32_t nb = n_padded / SCAN_TILE;
    k_scan_reduce<false><<<nb, SCAN_THREADS, 0, s>>>(in, partial, cond);
    k_scan_partials<<<1, 1024, 0, s>>>(partial, nb, cond);
    k_scan_down<false><<<nb, SCAN_THREADS, 0, s>>>(in, partial, out, n_padded, nb, cond);
}
void launch_scan_popc(const uint32_t* in, uint32_t* out, uint32_t* partial, uint32_t n_padded, cudaStream_t s) {
    const uint32_t nb = n_padded / SCAN_TILE;
    k_scan_reduce<true><<<nb, SCAN_THREADS, 0, s>>>(in, partial, nullptr);
    k_scan_partials<<<1, 1024, 0, s>>>(partial, nb, nullptr);
    k_scan_down<true><<<nb, SCAN_THREADS, 0, s>>>(in, partial, out, n_padded, nb, nullptr);
}
void launch_pack_keys(const uint8_t* sp, const int32_t* iz, const int32_t* ir, const float* pz, const float* pr,
                      int64_t n, int nz, int nr, uint32_t cell_base, uint32_t id0, uint32_t sp_max, uint32_t* key,
                      uint32_t* id, unsigned int* bad, int grid, cudaStream_t s) {
    k_pack_keys<<<grid, 256, 0, s>>>(sp, iz, ir, pz, pr, (long long)n, nz, nr, cell_base, id0, sp_max, key, id, bad);
}
void launch_species_count_all(const Particles& A, DevState* st, const KParams& P, unsigned long long* out, int grid,
                              cudaStream_t s) {
    if (P.nruns == 1) k_species_count1<<<grid, 256, 0, s>>>(A, st, out);
    else k_species_count_all<<<grid, 256, 0, s>>>(A, st, P, out);
}
void launch_density(const Particles& A, DevState* st, const KParams& P, int run, int species, long long* acc,
                    int grid, cudaStream_t s) {
    k_density<<<grid, 256, 0, s>>>(A, st, P, run, species, acc);
}
void launch_spectrum(const Particles& A, DevState* st, const KParams& P, int run, int species, double lo, double hi,
                     int nbins, unsigned long long* hist, int grid, cudaStream_t s) {
    k_spectrum<<<grid, 256, 0, s>>>(A, st, P, run, species, lo, hi, nbins, hist);
}

}  // namespace pd
