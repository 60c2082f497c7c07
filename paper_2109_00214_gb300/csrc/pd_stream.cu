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
// their new bin through one atomic cursor per bin, aggregated over the warp.
// With no previous order (after a load) everything is a mover and this is a
// plain counting sort.
//
// Both streaming kernels move four consecutive particles per thread with
// 128-bit loads issued before use.  Slot arrays are padded to a multiple of
// four.  Compiled with -fmad=false: every float operation is rounded on its
// own, in the order written.
#include "pd_internal.cuh"
#include "pd_kernels.h"
#include "pd_warp.cuh"

namespace pd {

template <typename T>
__device__ __forceinline__ T pick5(const T (&a)[NSP], int sp) {
    return sp == 0 ? a[0] : sp == 1 ? a[1] : sp == 2 ? a[2] : sp == 3 ? a[3] : a[4];
}

__device__ __forceinline__ float lane_of(const float4& v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }
__device__ __forceinline__ uint32_t lane_of(const uint4& v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }

// cell -> (iz, ir) without an integer division: float estimate, then fix
__device__ __forceinline__ void decode_cell(uint32_t cell, const KParams& P, int& iz, int& ir) {
    int q = (int)((float)cell * P.inv_nr);
    int r = (int)cell - q * P.nr;
    while (r < 0) {
        q -= 1;
        r += P.nr;
    }
    while (r >= P.nr) {
        q += 1;
        r -= P.nr;
    }
    iz = q;
    ir = r;
}

__device__ __forceinline__ int wrap(int i, int n) {
    if ((unsigned)i >= (unsigned)n) i = ((i % n) + n) % n;
    return i;
}

constexpr uint32_t NOBIN = 0xFFFFFFFFu;

template <bool RZ, bool FIELD>
__global__ void __launch_bounds__(256) k_push4(Particles A, const float2* __restrict__ E, long long* rho_e,
                                               long long* rho_h, uint32_t* out_cnt, uint32_t* in_cnt,
                                               uint32_t* mv, const uint32_t* __restrict__ old_off, uint32_t nbins,
                                               DevState* st, KParams P, PushConsts pc) {
    const uint32_t n = (uint32_t)st->n_slots;
    const uint32_t n_sorted = P.use_prev ? old_off[nbins] : 0u;
    const uint32_t nv = (n + 3u) >> 2;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    uint4* key4 = reinterpret_cast<uint4*>(A.key);
    float4* pz4 = reinterpret_cast<float4*>(A.pz);
    float4* pr4 = reinterpret_cast<float4*>(A.pr);
    float4* vz4 = reinterpret_cast<float4*>(A.vz);
    float4* vr4 = reinterpret_cast<float4*>(A.vr);
    float4* vt4 = reinterpret_cast<float4*>(A.vt);
    for (uint32_t g0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); g0 < nv; g0 += stride) {
        const uint32_t g = g0 + lane;
        const bool gv = g < nv;
        uint4 K = make_uint4(DEAD, DEAD, DEAD, DEAD);
        float4 Z = make_float4(0, 0, 0, 0), R = Z, VZ = Z, VR = Z, VT = Z;
        if (gv) {
            K = key4[g];
            Z = pz4[g];
            R = pr4[g];
            VZ = vz4[g];
            VR = vr4[g];
            if (RZ) VT = vt4[g];
        }
        uint32_t ko[4];
        float zo[4], ro[4], vzo[4], vro[4], vto[4];
        bool moved_any = false, key_changed = false;
        uint32_t nib = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t i = 4u * g + (uint32_t)q;
            const uint32_t key_in = (gv && i < n) ? lane_of(K, q) : DEAD;
            float pz = lane_of(Z, q), pr = lane_of(R, q);
            float vz = lane_of(VZ, q), vr = lane_of(VR, q), vt = lane_of(VT, q);
            ko[q] = lane_of(K, q);
            zo[q] = pz;
            ro[q] = pr;
            vzo[q] = vz;
            vro[q] = vr;
            vto[q] = vt;
            const bool live = key_in != DEAD;
            const int sp = (int)key_species(key_in);
            const uint32_t cell_in = key_cell(key_in);
            const bool in_sorted = live && i < n_sorted;
            const uint32_t old_bin = in_sorted ? key_sorted_species(key_in) * P.ncell + cell_in : NOBIN;
            uint32_t cell = cell_in;
            const bool move = live && (sp == SP_E || P.heavy_step);
            bool keep = live;
            int iz = 0, ir = 0;
            if (move) {
                moved_any = true;
                decode_cell(cell, P, iz, ir);
                const float qmdt = pick5(pc.qmdt, sp), dtz = pick5(pc.dtz, sp), dtr = pick5(pc.dtr, sp);
                if (FIELD) {
                    const float gz = 1.0f - pz, gr = 1.0f - pr;
                    const float w00 = gz * gr, w10 = pz * gr, w01 = gz * pr, w11 = pz * pr;
                    const float2 e00 = E[node_of(P, iz, ir)], e10 = E[node_of(P, iz + 1, ir)];
                    const float2 e01 = E[node_of(P, iz, ir + 1)], e11 = E[node_of(P, iz + 1, ir + 1)];
                    const float ez = ((w00 * e00.x + w10 * e10.x) + w01 * e01.x) + w11 * e11.x;
                    const float er = ((w00 * e00.y + w10 * e10.y) + w01 * e01.y) + w11 * e11.y;
                    vz = vz + qmdt * ez;
                    vr = vr + qmdt * er;
                }
                const float z = pz + vz * dtz;
                const float fz = floorf(z);
                int niz = iz + (int)fz;
                float npz = z - fz;
                if (npz >= 1.0f) npz = 0x1.fffffep-1f;
                int nir;
                float npr;
                int electrode = -1;
                if (RZ) {
                    const float x = ((float)ir + pr) + vr * dtr;
                    const float y = vt * dtr;
                    const float rr = sqrtf(x * x + y * y);
                    float c = 1.0f, s = 0.0f;
                    if (rr > 0.0f) {
                        c = x / rr;
                        s = y / rr;
                    }
                    const float nvr = c * vr + s * vt;
                    const float nvt = c * vt - s * vr;
                    vr = nvr;
                    vt = nvt;
                    const float fr = floorf(rr);
                    nir = (int)fr;
                    npr = rr - fr;
                    if (npr >= 1.0f) npr = 0x1.fffffep-1f;
                    if (niz < 0) electrode = 0;
                    else if (niz >= P.nz) electrode = 1;
                    else if (nir >= P.nr) electrode = 2;
                } else {
                    const float r = pr + vr * dtr;
                    const float fr = floorf(r);
                    nir = ir + (int)fr;
                    npr = r - fr;
                    if (npr >= 1.0f) npr = 0x1.fffffep-1f;
                    niz = wrap(niz, P.nz);
                    nir = wrap(nir, P.nr);
                }
                if (electrode >= 0) {
                    keep = false;
                    const double v2 = (double)vz * vz + (double)vr * vr + (double)vt * vt;
                    const double ke = P.weight * (0.5 * pick5(P.masses, sp) * v2);
                    atomicAdd(&st->ctr[C_ABS + electrode * NSP + sp], 1ull);
                    atomicAdd(&st->absorbed_energy[electrode], ke);
                    const double qw = (double)charge_of(sp) * 1.602176634e-19 * P.weight;
                    if (electrode == 1) atomicAdd(&st->anode_charge_step, qw);
                    if (electrode == 0) atomicAdd(&st->charge_cathode, qw);
                } else {
                    cell = (uint32_t)niz * (uint32_t)P.nr + (uint32_t)nir;
                    zo[q] = npz;
                    ro[q] = npr;
                    vzo[q] = vz;
                    vro[q] = vr;
                    vto[q] = vt;
                    iz = niz;
                    ir = nir;
                    pz = npz;
                    pr = npr;
                }
            }
            const uint32_t key = keep ? make_key((uint32_t)sp, cell) : DEAD;
            if (live) {
                key_changed |= key != key_in;
                ko[q] = key;
            }
            const uint32_t new_bin = keep ? (uint32_t)sp * P.ncell + cell : NOBIN;
            const bool mover = in_sorted && new_bin != old_bin;
            const bool in_mover = keep && (!in_sorted || new_bin != old_bin);
            nib |= (mover ? 1u : 0u) << q;
            if (mover) atomicAdd(&out_cnt[old_bin], 1u);
            warp_count(in_cnt, new_bin, in_mover);
            const int zq = charge_of(sp);
            const bool dep = move && keep && zq != 0;
            // electrons and heavies deposit into separate grids (heavies are
            // held between their sub-cycled pushes)
            if (__any_sync(FULL_MASK, dep)) {
                long long* rho = sp == SP_E ? rho_e : rho_h;
                warp_deposit(rho, P, key, iz, ir, pz, pr, zq, dep);
            }
        }
        // mover bits: particle 4g+q is bit (4g+q) % 32 of word (4g+q) / 32
        uint32_t word = nib << (4 * (lane & 7));
        word |= __shfl_xor_sync(FULL_MASK, word, 1);
        word |= __shfl_xor_sync(FULL_MASK, word, 2);
        word |= __shfl_xor_sync(FULL_MASK, word, 4);
        if ((lane & 7) == 0 && gv) mv[(g0 >> 3) + (lane >> 3)] = word;
        if (gv && (moved_any || key_changed)) {
            key4[g] = make_uint4(ko[0], ko[1], ko[2], ko[3]);
            if (moved_any) {
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

// movers strictly before slot p (p < n_sorted)
__device__ __forceinline__ uint32_t movers_before(const uint32_t* __restrict__ mv, const uint32_t* __restrict__ mvx,
                                                  uint32_t p) {
    const uint32_t w = p >> 5;
    return mvx[w] + (uint32_t)__popc(mv[w] & ((1u << (p & 31u)) - 1u));
}

__global__ void __launch_bounds__(256) k_scatter4(Particles A, Particles B, const uint32_t* __restrict__ old_off,
                                                  const uint32_t* __restrict__ new_off,
                                                  const uint32_t* __restrict__ stay, uint32_t* in_cnt,
                                                  const uint32_t* __restrict__ mv, const uint32_t* __restrict__ mvx,
                                                  uint32_t nbins, DevState* st, KParams P) {
    const uint32_t n = (uint32_t)st->n_slots;
    const uint32_t n_sorted = P.use_prev ? old_off[nbins] : 0u;
    const uint32_t nv = (n + 3u) >> 2;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    const unsigned lt = lanemask_lt();
    for (uint32_t g0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); g0 < nv; g0 += stride) {
        const uint32_t g = g0 + lane;
        const bool gv = g < nv;
        uint4 K = make_uint4(DEAD, DEAD, DEAD, DEAD), ID = K;
        float4 Z = make_float4(0, 0, 0, 0), R = Z, VZ = Z, VR = Z, VT = Z;
        uint32_t mw = 0, mx = 0;
        if (gv) {
            K = reinterpret_cast<const uint4*>(A.key)[g];
            Z = reinterpret_cast<const float4*>(A.pz)[g];
            R = reinterpret_cast<const float4*>(A.pr)[g];
            VZ = reinterpret_cast<const float4*>(A.vz)[g];
            VR = reinterpret_cast<const float4*>(A.vr)[g];
            VT = reinterpret_cast<const float4*>(A.vt)[g];
            ID = reinterpret_cast<const uint4*>(A.id)[g];
            if (4u * g < n_sorted) {
                mw = mv[g >> 3];
                mx = mvx[g >> 3];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t i = 4u * g + (uint32_t)q;
            const uint32_t key = (gv && i < n) ? lane_of(K, q) : DEAD;
            const bool live = key != DEAD;
            const uint32_t b = live ? key_species(key) * P.ncell + key_cell(key) : 0u;
            const bool stayer = live && i < n_sorted && !((mw >> (i & 31u)) & 1u);
            const bool mover = live && !stayer;
            uint32_t slot = 0;
            if (stayer) {
                const uint32_t o = old_off[b];
                const uint32_t before = mx + (uint32_t)__popc(mw & ((1u << (i & 31u)) - 1u));
                slot = new_off[b] + (i - o) - (before - movers_before(mv, mvx, o));
            }
            const unsigned m = __ballot_sync(FULL_MASK, mover);
            if (mover) {
                const unsigned grp = __match_any_sync(m, b);
                const int leader = __ffs(grp) - 1;
                const uint32_t cnt = (uint32_t)__popc(grp);
                uint32_t old = 0;
                if (lane == leader) old = atomicSub(&in_cnt[b], cnt);
                old = __shfl_sync(grp, old, leader);
                slot = new_off[b] + stay[b] + old - cnt + (uint32_t)__popc(grp & lt);
            }
            if (live && slot >= n) {        // inconsistent bookkeeping: report, never write out of range
                set_error(st, ERR_BOUNDS);
                continue;
            }
            if (live) {
                B.key[slot] = key;
                B.pz[slot] = lane_of(Z, q);
                B.pr[slot] = lane_of(R, q);
                B.vz[slot] = lane_of(VZ, q);
                B.vr[slot] = lane_of(VR, q);
                B.vt[slot] = lane_of(VT, q);
                B.id[slot] = lane_of(ID, q);
            }
        }
    }
}

void launch_push(const Particles& A, const float2* E, long long* rho_e, long long* rho_h, uint32_t* out_cnt,
                 uint32_t* in_cnt, uint32_t* mv, const uint32_t* old_off, uint32_t nbins, DevState* st,
                 const KParams& P, const PushConsts& pc, int grid, cudaStream_t s) {
    const bool rz = P.geom == 0, field = P.field_on != 0;
#define PD_PUSH_ARGS A, E, rho_e, rho_h, out_cnt, in_cnt, mv, old_off, nbins, st, P, pc
    if (rz && field) k_push4<true, true><<<grid, 256, 0, s>>>(PD_PUSH_ARGS);
    else if (rz) k_push4<true, false><<<grid, 256, 0, s>>>(PD_PUSH_ARGS);
    else if (field) k_push4<false, true><<<grid, 256, 0, s>>>(PD_PUSH_ARGS);
    else k_push4<false, false><<<grid, 256, 0, s>>>(PD_PUSH_ARGS);
#undef PD_PUSH_ARGS
}

void launch_bincount(const uint32_t* old_off, uint32_t* out_cnt, const uint32_t* in_cnt, uint32_t* cnt,
                     uint32_t* stay, uint32_t nbins_pad, int use_prev, int grid, cudaStream_t s) {
    k_bincount<<<grid, 256, 0, s>>>(old_off, out_cnt, in_cnt, cnt, stay, nbins_pad, use_prev);
}

void launch_scatter(const Particles& A, const Particles& B, const uint32_t* old_off, const uint32_t* new_off,
                    const uint32_t* stay, uint32_t* in_cnt, const uint32_t* mv, const uint32_t* mvx, uint32_t nbins,
                    DevState* st, const KParams& P, int grid, cudaStream_t s) {
    k_scatter4<<<grid, 256, 0, s>>>(A, B, old_off, new_off, stay, in_cnt, mv, mvx, nbins, st, P);
}

}  // namespace pd
