// pd_stream.cu -- the particle-streaming kernels of the step.
//
//   k_push4     Newton push (Sec. 2.1) with the field gathered by the CIC
//               weights of Eq. (10), r-z rotation or periodic wrap, absorbing
//               walls, fused with the fixed-point CIC deposit of Eq. (9)-(10)
//               and the bookkeeping of the cell sort.
//   k_bincount  new bin counts = sorted counts - movers out + movers in.
//   k_scatter4  the sort itself, A -> B in (species, cell) order.
//
// The sort exploits that a step moves few particles out of their (species,
// cell) bin.  Slots [0, n_sorted) hold the previous step's sorted order.  A
// particle there that stays in its bin ("stayer") goes to
//     new_off[b] + (p - old_off[b]) - (movers in [old_off[b], p)),
// computed from a bit mask of movers and its popcount prefix: no atomics, and
// the stayers of a warp land on consecutive slots.  Movers, spawned and
// injected particles (slots >= n_sorted) take slots after the stayers of
// their new bin through one atomic cursor per bin.  With no previous order
// (after a load) everything is a mover and this is a plain counting sort.
//
// Each thread moves four consecutive particles with 128-bit loads issued
// before use.  Sorted input means the four usually share a cell, so counts,
// slot claims and deposited charge are merged over runs of equal keys inside
// the thread (no warp-wide collectives on the common path), and the push
// arithmetic is done for all four and selected, without divergent branches.
// Slot arrays are padded to a multiple of four.  Compiled with -fmad=false:
// every float operation is rounded on its own, in the order written.
#include "pd_internal.cuh"
#include "pd_kernels.h"
#include "pd_warp.cuh"

namespace pd {

// a[sp] without dynamic indexing (kernel parameters)
template <typename T>
__device__ __forceinline__ T pick_sp(const T (&a)[NSP], int sp) {
    T r = a[0];
#pragma unroll
    for (int k = 1; k < NSP; ++k) r = sp == k ? a[k] : r;
    return r;
}

__device__ __forceinline__ float lane_of(const float4& v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }
__device__ __forceinline__ uint32_t lane_of(const uint4& v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }

// local cell -> (iz, ir) without an integer division: the float estimate is
// within one of the quotient for cell < 2^24 and nr >= 2; fix it without branches
__device__ __forceinline__ void decode_cell(uint32_t cell, int nr, float inv_nr, int& iz, int& ir) {
    int q = (int)((float)cell * inv_nr);
    int r = (int)cell - q * nr;
    const int lo = r < 0 ? 1 : 0, hi = r >= nr ? 1 : 0;
    q += hi - lo;
    r += (lo - hi) * nr;
    iz = q;
    ir = r;
}

// periodic wrap of an index that moved by at most one period
__device__ __forceinline__ int wrap1(int i, int n) {
    i += i < 0 ? n : 0;
    i -= i >= n ? n : 0;
    return i;
}

// Runs of equal keys among the "on" entries of four consecutive particles:
// link[q] = particle q continues the run of q-1; len[q] = length of the run
// that starts at q (0 if q does not start one).
__device__ __forceinline__ void runs4(const bool (&on)[4], const uint32_t (&key)[4], bool (&link)[4],
                                      uint32_t (&len)[4]) {
    link[0] = false;
#pragma unroll
    for (int q = 1; q < 4; ++q) link[q] = on[q] && on[q - 1] && key[q] == key[q - 1];
    const uint32_t c3 = 0, c2 = link[3] ? 1u + c3 : 0u, c1 = link[2] ? 1u + c2 : 0u, c0 = link[1] ? 1u + c1 : 0u;
    const uint32_t c[4] = {c0, c1, c2, c3};
#pragma unroll
    for (int q = 0; q < 4; ++q) len[q] = (on[q] && !link[q]) ? 1u + c[q] : 0u;
}

constexpr uint32_t NOBIN = 0xFFFFFFFFu;

// per-species constant: shared-memory table (ensembles) or kernel parameter
// (one run, selected without dynamic indexing)
template <bool MULTI>
__device__ __forceinline__ float spc(const float (&a)[NSP], int sp) {
    return MULTI ? a[sp] : pick_sp(a, sp);
}
// a constant that depends only on electron vs heavy (the time step ratios:
// every heavy species moves with the heavy step)
template <bool MULTI>
__device__ __forceinline__ float spc_eh(const float (&a)[NSP], int sp) {
    return MULTI ? a[sp] : (sp == SP_E ? a[0] : a[1]);
}

template <bool RZ, bool FIELD, bool MULTI>
__global__ void __launch_bounds__(256, (RZ || FIELD) ? 3 : 4) k_push4(Particles A, const float2* __restrict__ E, long long* rho_e,
                                               long long* rho_h, uint32_t* out_cnt, uint32_t* in_cnt,
                                               uint32_t* mv, const uint32_t* __restrict__ old_off, uint32_t nbins,
                                               DevState* st, KParams P) {
    __shared__ RunInfo s_runs[MULTI ? MAX_RUNS_SMEM : 1];
    if (MULTI) {
        for (int r = threadIdx.x; r < P.nruns; r += blockDim.x) s_runs[r] = P.runs[r];
        __syncthreads();
    }
    const uint32_t n = (uint32_t)st->n_slots;
    const uint32_t n_sorted = P.use_prev ? old_off[nbins] : 0u;
    const uint32_t nv = (n + 3u) >> 2;
    const uint32_t stride = gridDim.x * blockDim.x;
    const int geom = RZ ? 0 : 1;
    uint4* key4 = reinterpret_cast<uint4*>(A.key);
    float4* pz4 = reinterpret_cast<float4*>(A.pz);
    float4* pr4 = reinterpret_cast<float4*>(A.pr);
    float4* vz4 = reinterpret_cast<float4*>(A.vz);
    float4* vr4 = reinterpret_cast<float4*>(A.vr);
    float4* vt4 = reinterpret_cast<float4*>(A.vt);
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g - threadIdx.x % 32u < nv; g += stride) {
        const bool gv = g < nv;
        uint4 K = make_uint4(DEAD, DEAD, DEAD, DEAD);
        float4 Z = make_float4(0, 0, 0, 0), R4 = Z, VZ = Z, VR = Z, VT = Z;
        if (gv) {
            K = key4[g];
            Z = pz4[g];
            R4 = pr4[g];
            VZ = vz4[g];
            VR = vr4[g];
            if (RZ) VT = vt4[g];
        }
        uint32_t ko[4], key[4], newbin[4], oldbin[4];
        float zo[4], ro[4], vzo[4], vro[4], vto[4];
        int sp_[4], iz_[4], ir_[4], wall_[4], run_[4];
        bool mover[4], inmv[4], dep[4], absd[4];
        uint32_t flags = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t i = 4u * g + (uint32_t)q;
            const uint32_t key_in = (gv && i < n) ? lane_of(K, q) : DEAD;
            const float pz = lane_of(Z, q), pr = lane_of(R4, q);
            float vz = lane_of(VZ, q), vr = lane_of(VR, q), vt = lane_of(VT, q);
            const bool live = key_in != DEAD;
            const int sp = live ? (int)key_species(key_in) : 0;
            const uint32_t gcell_in = live ? key_cell(key_in) : 0u;
            const int r = live ? run_of(P, gcell_in) : 0;
            const RunInfo& RI = MULTI ? s_runs[r] : P.run0;
            const bool in_sorted = live && i < n_sorted;
            oldbin[q] = in_sorted ? key_sorted_species(key_in) * P.ncell + gcell_in : NOBIN;
            const bool move = live && (sp == SP_E || P.heavy_step);
            const uint32_t lcell = move ? gcell_in - RI.cell_base : 0u;   // dead lanes read a valid node
            int iz, ir;
            decode_cell(lcell, RI.nr, RI.inv_nr, iz, ir);
            const float qmdt = spc<MULTI>(RI.qmdt, sp), dtz = spc_eh<MULTI>(RI.dtz, sp), dtr = spc_eh<MULTI>(RI.dtr, sp);
            if (FIELD) {
                const float gz = 1.0f - pz, gr = 1.0f - pr;
                const float w00 = gz * gr, w10 = pz * gr, w01 = gz * pr, w11 = pz * pr;
                const float2 e00 = E[node_of(RI, geom, iz, ir)], e10 = E[node_of(RI, geom, iz + 1, ir)];
                const float2 e01 = E[node_of(RI, geom, iz, ir + 1)], e11 = E[node_of(RI, geom, iz + 1, ir + 1)];
                const float ez = ((w00 * e00.x + w10 * e10.x) + w01 * e01.x) + w11 * e11.x;
                const float er = ((w00 * e00.y + w10 * e10.y) + w01 * e01.y) + w11 * e11.y;
                vz = vz + qmdt * ez;
                vr = vr + qmdt * er;
            }
            const float z = pz + vz * dtz;
            const float fz = floorf(z);
            int niz = iz + (int)fz;
            float npz = z - fz;
            npz = npz >= 1.0f ? 0x1.fffffep-1f : npz;
            int nir;
            float npr;
            bool out = false;
            if (RZ) {
                const float x = ((float)ir + pr) + vr * dtr;
                const float y = vt * dtr;
                const float rr = sqrtf(x * x + y * y);
                const bool pos = rr > 0.0f;
                const float c = pos ? x / rr : 1.0f, s = pos ? y / rr : 0.0f;
                const float nvr = c * vr + s * vt;
                const float nvt = c * vt - s * vr;
                vr = nvr;
                vt = nvt;
                const float fr = floorf(rr);
                nir = (int)fr;
                npr = rr - fr;
                npr = npr >= 1.0f ? 0x1.fffffep-1f : npr;
                out = niz < 0 || niz >= RI.nz || nir >= RI.nr;
                // cathode (z = 0) before anode (z = L) before the outer wall (r = R)
                wall_[q] = niz < 0 ? 0 : (niz >= RI.nz ? 1 : 2);
            } else {
                wall_[q] = 0;
                const float rr = pr + vr * dtr;
                const float fr = floorf(rr);
                nir = ir + (int)fr;
                npr = rr - fr;
                npr = npr >= 1.0f ? 0x1.fffffep-1f : npr;
                // a particle crosses at most one period per step (|v dt| < one domain)
                niz = wrap1(niz, RI.nz);
                nir = wrap1(nir, RI.nr);
            }
            const bool absorbed = move && out;
            const bool kp = live && !absorbed;
            const uint32_t gcell =
                move ? RI.cell_base + (uint32_t)niz * (uint32_t)RI.nr + (uint32_t)nir : gcell_in;
            const uint32_t k = kp ? make_key((uint32_t)sp, gcell) : DEAD;
            const uint32_t nb = kp ? (uint32_t)sp * P.ncell + gcell : NOBIN;
            const bool mvq = in_sorted && nb != oldbin[q];
            const bool inq = kp && (!in_sorted || nb != oldbin[q]);
            const bool mk = move && kp;
            ko[q] = live ? k : lane_of(K, q);
            key[q] = k;
            newbin[q] = nb;
            mover[q] = mvq;
            inmv[q] = inq;
            absd[q] = absorbed;
            zo[q] = mk ? npz : pz;
            ro[q] = (mk || absorbed) ? npr : pr;           // an absorbed particle keeps its impact r
            vzo[q] = move ? vz : lane_of(VZ, q);
            vro[q] = move ? vr : lane_of(VR, q);
            vto[q] = move ? vt : lane_of(VT, q);
            sp_[q] = sp;
            run_[q] = r;
            iz_[q] = mk ? niz : iz;
            ir_[q] = (mk || absorbed) ? nir : ir;
            dep[q] = mk && charge_of(sp) != 0;
            // 16: the particle moved (new position); 32: its key changed (new
            // bin, absorbed, or converted in the last collisions)
            flags |= (absorbed ? 1u : 0u) | (mvq ? 2u : 0u) | (inq ? 4u : 0u) | (dep[q] ? 8u : 0u) |
                     (mk ? 16u : 0u) | ((live && k != lane_of(K, q)) ? 32u : 0u);
        }
        const uint32_t wflags = __reduce_or_sync(FULL_MASK, flags);
        if (RZ && (wflags & 1u)) {  // absorbed at an electrode or the outer wall: ledgers
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!absd[q]) continue;
                const int sp = sp_[q];
                const int electrode = wall_[q];
                RunState& rs = P.rs[run_[q]];
                const double v2 = (double)vzo[q] * vzo[q] + (double)vro[q] * vro[q] + (double)vto[q] * vto[q];
                const double w = MULTI ? s_runs[run_[q]].weight : P.run0.weight;
                const double ke = w * (0.5 * pick_sp(P.masses, sp) * v2);
                atomicAdd(&rs.ctr[C_ABS + electrode * NSP + sp], 1ull);
                atomicAdd(&rs.absorbed_energy[electrode], ke);
                const double qw = (double)charge_of(sp) * 1.602176634e-19 * w;
                if (electrode == 1) atomicAdd(&rs.anode_charge_step, qw);
                if (electrode == 0) atomicAdd(&rs.charge_cathode, qw);
                // an ion arriving at an electrode inside the outer radius sputters
                // floor(Y(E) + R) atoms (emitted by k_sputter)
                const RunInfo& RI = MULTI ? s_runs[run_[q]] : P.run0;
                if (P.sputter && electrode < 2 && charge_of(sp) > 0 && ir_[q] < RI.nr) {
                    const float E = (float)((0.5 * pick_sp(P.masses, sp) * v2) / 1.602176634e-19);
                    const float Y = xs_lookup(P.xsE, P.ytab, E);
                    const uint32_t id = A.id[4u * g + (uint32_t)q];
                    Stream rs_(id, st->step, SID_SPUT, RI.seed, RI.run);
                    const uint32_t nsp = (uint32_t)floorf(Y + rs_.u01());
                    if (nsp) {
                        const uint32_t x = atomicAdd(&st->n_sput, 1u);
                        if (x < P.squeue_cap)
                            P.squeue[x] = SputRec{id, ((uint32_t)run_[q] << 1) | (uint32_t)electrode, (uint32_t)ir_[q],
                                                  ro[q], nsp};
                        else
                            set_error(st, ERR_CAPACITY);
                    }
                }
            }
        }
        if (wflags & 2u) {          // movers out of their sorted bin
            uint32_t nib = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (mover[q]) atomicAdd(&out_cnt[oldbin[q]], 1u);
                nib |= (mover[q] ? 1u : 0u) << q;
            }
            if (nib) atomicOr(&mv[g >> 3], nib << (4u * (g & 7u)));
        }
        if (wflags & 4u) {          // movers into their new bin (all particles after a load)
            bool link[4];
            uint32_t len[4];
            runs4(inmv, newbin, link, len);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (len[q]) atomicAdd(&in_cnt[newbin[q]], len[q]);
        }
        if (wflags & 8u) {          // fixed-point CIC deposit, merged over runs of one key
            bool link[4];
            uint32_t len[4];
            runs4(dep, key, link, len);
            unsigned long long W[4][4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t wz = __float2uint_rn(zo[q] * 65536.0f);
                const uint32_t wr = __float2uint_rn(ro[q] * 65536.0f);
                const unsigned long long az = 65536u - wz, ar = 65536u - wr;
                W[q][0] = dep[q] ? az * ar : 0ull;
                W[q][1] = dep[q] ? (unsigned long long)wz * ar : 0ull;
                W[q][2] = dep[q] ? az * (unsigned long long)wr : 0ull;
                W[q][3] = dep[q] ? (unsigned long long)wz * wr : 0ull;
            }
            // accumulate each run into its first particle (runs are contiguous)
#pragma unroll
            for (int q = 3; q >= 1; --q)
                if (link[q])
#pragma unroll
                    for (int c = 0; c < 4; ++c) W[q - 1][c] += W[q][c];
            // r-z plumes hold cells of thousands of particles: when all 128
            // particles of the warp deposit into one cell, the warp sums the
            // four corner weights and issues four atomics instead of 128
            bool one_cell_warp = false;
            if constexpr (RZ) {
                const uint32_t k0 = __shfl_sync(FULL_MASK, key[0], 0);
                const bool one_cell = dep[0] && dep[1] && dep[2] && dep[3] && key[0] == k0 && key[1] == k0 &&
                                      key[2] == k0 && key[3] == k0;
                one_cell_warp = __all_sync(FULL_MASK, one_cell);
            }
            if (one_cell_warp) {
                unsigned long long Ws[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    Ws[c] = W[0][c];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) Ws[c] += __shfl_down_sync(FULL_MASK, Ws[c], o);
                }
                if ((threadIdx.x & 31u) == 0) {
                    const long long zq = charge_of(sp_[0]);
                    long long* rho = sp_[0] == SP_E ? rho_e : rho_h;
                    const RunInfo& RI = MULTI ? s_runs[run_[0]] : P.run0;
                    const int iz = iz_[0], ir = ir_[0];
                    atomicAdd((unsigned long long*)&rho[node_of(RI, geom, iz, ir)],
                              (unsigned long long)(zq * (long long)Ws[0]));
                    atomicAdd((unsigned long long*)&rho[node_of(RI, geom, iz + 1, ir)],
                              (unsigned long long)(zq * (long long)Ws[1]));
                    atomicAdd((unsigned long long*)&rho[node_of(RI, geom, iz, ir + 1)],
                              (unsigned long long)(zq * (long long)Ws[2]));
                    atomicAdd((unsigned long long*)&rho[node_of(RI, geom, iz + 1, ir + 1)],
                              (unsigned long long)(zq * (long long)Ws[3]));
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (!len[q]) continue;
                    const long long zq = charge_of(sp_[q]);
                    long long* rho = sp_[q] == SP_E ? rho_e : rho_h;
                    const RunInfo& RI = MULTI ? s_runs[run_[q]] : P.run0;
                    const int iz = iz_[q], ir = ir_[q];
                    atomicAdd((unsigned long long*)&rho[node_of(RI, geom, iz, ir)],
                              (unsigned long long)(zq * (long long)W[q][0]));
                    atomicAdd((unsigned long long*)&rho[node_of(RI, geom, iz + 1, ir)],
                              (unsigned long long)(zq * (long long)W[q][1]));
                    atomicAdd((unsigned long long*)&rho[node_of(RI, geom, iz, ir + 1)],
                              (unsigned long long)(zq * (long long)W[q][2]));
                    atomicAdd((unsigned long long*)&rho[node_of(RI, geom, iz + 1, ir + 1)],
                              (unsigned long long)(zq * (long long)W[q][3]));
                }
            }
        }
        // write back only what changed: most keys do not change in a step
        if (gv && (flags & 32u)) key4[g] = make_uint4(ko[0], ko[1], ko[2], ko[3]);
        if (gv && (flags & 16u)) {
            pz4[g] = make_float4(zo[0], zo[1], zo[2], zo[3]);
            pr4[g] = make_float4(ro[0], ro[1], ro[2], ro[3]);
            if (FIELD || RZ) {
                vz4[g] = make_float4(vzo[0], vzo[1], vzo[2], vzo[3]);
                vr4[g] = make_float4(vro[0], vro[1], vro[2], vro[3]);
            }
            if (RZ) vt4[g] = make_float4(vto[0], vto[1], vto[2], vto[3]);
        }
    }
}

// cnt[b] = (sorted count of b) - out[b] + in[b]; stay[b] = sorted - out; out := 0
__global__ void __launch_bounds__(256) k_bincount(const uint32_t* __restrict__ old_off, uint32_t* out_cnt,
                                                  const uint32_t* __restrict__ in_cnt, uint32_t* cnt, uint32_t* stay,
                                                  uint32_t nbins_pad, int use_prev) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins_pad; b += gridDim.x * blockDim.x) {
        const uint32_t sorted = use_prev ? old_off[b + 1] - old_off[b] : 0u;
        const uint32_t s = sorted - out_cnt[b];
        stay[b] = s;
        cnt[b] = s + in_cnt[b];
        out_cnt[b] = 0u;
    }
}

// movers strictly before slot p (p <= n_sorted)
__device__ __forceinline__ uint32_t movers_before(const uint32_t* __restrict__ mv, const uint32_t* __restrict__ mvx,
                                                  uint32_t p) {
    const uint32_t w = p >> 5;
    return mvx[w] + (uint32_t)__popc(mv[w] & ((1u << (p & 31u)) - 1u));
}

// dlt[b] = new_off[b] - old_off[b] + (movers before old_off[b]): a stayer of
// bin b at old slot i goes to dlt[b] + i - (movers before i)
__global__ void __launch_bounds__(256) k_bin_delta(const uint32_t* __restrict__ old_off,
                                                   const uint32_t* __restrict__ new_off,
                                                   const uint32_t* __restrict__ mv, const uint32_t* __restrict__ mvx,
                                                   uint32_t* dlt, uint32_t nbins) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        const uint32_t o = old_off[b];
        dlt[b] = new_off[b] - o + movers_before(mv, mvx, o);
    }
}

// Staging window of the scatter: a block's stayers land on a nearly
// contiguous range of slots (its own particles plus the movers other blocks
// insert between its bins); stayers within SCATTER_WIN slots of the block's
// first one go through shared memory and are written out in slot order.
constexpr int SCATTER_THREADS = 256;
constexpr uint32_t SCATTER_WIN = 1536;

__global__ void __launch_bounds__(SCATTER_THREADS, 4) k_scatter4(Particles A, Particles B,
                                                              const uint32_t* __restrict__ old_off,
                                                              const uint32_t* __restrict__ new_off,
                                                              const uint32_t* __restrict__ stay,
                                                              const uint32_t* __restrict__ dlt, uint32_t* in_cnt,
                                                              const uint32_t* __restrict__ mv,
                                                              const uint32_t* __restrict__ mvx, uint32_t nbins,
                                                              DevState* st, KParams P) {
    __shared__ uint32_t s_key[SCATTER_WIN], s_id[SCATTER_WIN];
    __shared__ float s_pz[SCATTER_WIN], s_pr[SCATTER_WIN], s_vz[SCATTER_WIN], s_vr[SCATTER_WIN], s_vt[SCATTER_WIN];
    __shared__ uint32_t s_base;
    const uint32_t n = (uint32_t)st->n_slots;
    const uint32_t n_sorted = P.use_prev ? old_off[nbins] : 0u;
    const uint32_t nv = (n + 3u) >> 2;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = threadIdx.x; k < SCATTER_WIN; k += blockDim.x) s_key[k] = DEAD;
    if (threadIdx.x == 0) s_base = 0xFFFFFFFFu;
    __syncthreads();
    for (uint32_t g0 = blockIdx.x * blockDim.x; g0 < nv; g0 += stride) {
        const uint32_t g = g0 + threadIdx.x;
        const bool gv = g < nv;
        uint4 K = make_uint4(DEAD, DEAD, DEAD, DEAD), ID = K;
        float4 Z = make_float4(0, 0, 0, 0), R = Z, VZ = Z, VR = Z, VT = Z;
        if (gv) {
            K = reinterpret_cast<const uint4*>(A.key)[g];
            Z = reinterpret_cast<const float4*>(A.pz)[g];
            R = reinterpret_cast<const float4*>(A.pr)[g];
            VZ = reinterpret_cast<const float4*>(A.vz)[g];
            VR = reinterpret_cast<const float4*>(A.vr)[g];
            VT = reinterpret_cast<const float4*>(A.vt)[g];
            ID = reinterpret_cast<const uint4*>(A.id)[g];
        }
        const bool sorted_part = gv && 4u * g < n_sorted;
        const uint32_t mw = sorted_part ? mv[g >> 3] : 0u;
        const uint32_t mx = sorted_part ? mvx[g >> 3] : 0u;
        uint32_t key[4], bin[4], slot[4];
        bool live[4], mover[4], stays[4];
        bool any_mover = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t i = 4u * g + (uint32_t)q;
            key[q] = (gv && i < n) ? lane_of(K, q) : DEAD;
            live[q] = key[q] != DEAD;
            bin[q] = live[q] ? key_species(key[q]) * P.ncell + key_cell(key[q]) : 0u;
            const bool stayer = live[q] && i < n_sorted && !((mw >> (i & 31u)) & 1u);
            mover[q] = live[q] && !stayer;
            stays[q] = stayer;
            any_mover |= mover[q];
            slot[q] = 0;
            if (stayer) {
                // slot = new_off - old_off + (movers before old_off) + i - (movers before i), the
                // bin's part precomputed in dlt
                const uint32_t before = mx + (uint32_t)__popc(mw & ((1u << (i & 31u)) - 1u));
                slot[q] = dlt[bin[q]] + i - before;

            }
        }
        if (any_mover) {            // claim slots after the stayers, one atomic per run of one bin
            bool link[4];
            uint32_t len[4];
            runs4(mover, bin, link, len);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (len[q]) {
                    const uint32_t old = atomicSub(&in_cnt[bin[q]], len[q]);
                    if (old < len[q]) set_error(st, ERR_BOUNDS);      // more movers than counted
                    slot[q] = new_off[bin[q]] + stay[bin[q]] + old - len[q];
                } else if (link[q]) {
                    slot[q] = (q > 0 ? slot[q > 0 ? q - 1 : 0] : 0u) + 1u;
                }
            }
        }
        // the block's first stayer slot anchors the staging window
        uint32_t my_min = 0xFFFFFFFFu;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (stays[q] && slot[q] < my_min) my_min = slot[q];
        my_min = __reduce_min_sync(FULL_MASK, my_min);
        if ((threadIdx.x & 31) == 0 && my_min != 0xFFFFFFFFu) atomicMin(&s_base, my_min);
        __syncthreads();
        const uint32_t base = s_base;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!live[q]) continue;
            if (slot[q] >= n) {     // inconsistent bookkeeping: report, never write out of range
                set_error(st, ERR_BOUNDS);
                continue;
            }
            const uint32_t s = slot[q];
            const uint32_t w = s - base;
            if (stays[q] && w < SCATTER_WIN) {
                s_key[w] = key[q];
                s_pz[w] = lane_of(Z, q);
                s_pr[w] = lane_of(R, q);
                s_vz[w] = lane_of(VZ, q);
                s_vr[w] = lane_of(VR, q);
                s_vt[w] = lane_of(VT, q);
                s_id[w] = lane_of(ID, q);
            } else {
                B.key[s] = key[q];
                B.pz[s] = lane_of(Z, q);
                B.pr[s] = lane_of(R, q);
                B.vz[s] = lane_of(VZ, q);
                B.vr[s] = lane_of(VR, q);
                B.vt[s] = lane_of(VT, q);
                B.id[s] = lane_of(ID, q);
            }
        }
        __syncthreads();
        // write the window out in slot order: consecutive threads, consecutive slots
        if (base != 0xFFFFFFFFu) {
            for (uint32_t e = threadIdx.x; e < SCATTER_WIN; e += blockDim.x) {
                const uint32_t k = s_key[e];
                if (k == DEAD) continue;
                const uint32_t s = base + e;
                B.key[s] = k;
                B.pz[s] = s_pz[e];
                B.pr[s] = s_pr[e];
                B.vz[s] = s_vz[e];
                B.vr[s] = s_vr[e];
                B.vt[s] = s_vt[e];
                B.id[s] = s_id[e];
                s_key[e] = DEAD;
            }
        }
        if (threadIdx.x == 0) s_base = 0xFFFFFFFFu;
        __syncthreads();
    }
}

void launch_push(const Particles& A, const float2* E, long long* rho_e, long long* rho_h, uint32_t* out_cnt,
                 uint32_t* in_cnt, uint32_t* mv, const uint32_t* old_off, uint32_t nbins, DevState* st,
                 const KParams& P, int grid, cudaStream_t s) {
    const bool rz = P.geom == 0, field = P.field_on != 0;
#define PD_PUSH_ARGS A, E, rho_e, rho_h, out_cnt, in_cnt, mv, old_off, nbins, st, P
    if (P.nruns > 1) {
        if (rz && field) k_push4<true, true, true><<<grid, 256, 0, s>>>(PD_PUSH_ARGS);
        else if (rz) k_push4<true, false, true><<<grid, 256, 0, s>>>(PD_PUSH_ARGS);
        else if (field) k_push4<false, true, true><<<grid, 256, 0, s>>>(PD_PUSH_ARGS);
        else k_push4<false, false, true><<<grid, 256, 0, s>>>(PD_PUSH_ARGS);
    } else {
        if (rz && field) k_push4<true, true, false><<<grid, 256, 0, s>>>(PD_PUSH_ARGS);
        else if (rz) k_push4<true, false, false><<<grid, 256, 0, s>>>(PD_PUSH_ARGS);
        else if (field) k_push4<false, true, false><<<grid, 256, 0, s>>>(PD_PUSH_ARGS);
        else k_push4<false, false, false><<<grid, 256, 0, s>>>(PD_PUSH_ARGS);
    }
#undef PD_PUSH_ARGS
}

void launch_bincount(const uint32_t* old_off, uint32_t* out_cnt, const uint32_t* in_cnt, uint32_t* cnt,
                     uint32_t* stay, uint32_t nbins_pad, int use_prev, int grid, cudaStream_t s) {
    k_bincount<<<grid, 256, 0, s>>>(old_off, out_cnt, in_cnt, cnt, stay, nbins_pad, use_prev);
}

void launch_bin_delta(const uint32_t* old_off, const uint32_t* new_off, const uint32_t* mv, const uint32_t* mvx,
                      uint32_t* dlt, uint32_t nbins, int grid, cudaStream_t s) {
    k_bin_delta<<<grid, 256, 0, s>>>(old_off, new_off, mv, mvx, dlt, nbins);
}

void launch_scatter(const Particles& A, const Particles& B, const uint32_t* old_off, const uint32_t* new_off,
                    const uint32_t* stay, const uint32_t* dlt, uint32_t* in_cnt, const uint32_t* mv,
                    const uint32_t* mvx, uint32_t nbins, DevState* st, const KParams& P, int grid, cudaStream_t s) {
    k_scatter4<<<grid, SCATTER_THREADS, 0, s>>>(A, B, old_off, new_off, stay, dlt, in_cnt, mv, mvx, nbins, st, P);
}

}  // namespace pd
