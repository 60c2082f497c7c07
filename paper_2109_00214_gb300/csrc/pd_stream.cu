// pd_stream.cu -- the two particle-streaming kernels of the step.
//
//   k_push4     Newton push (Sec. 2.1) with the field gathered by the CIC
//               weights of Eq. (10), r-z rotation or periodic wrap, absorbing
//               walls, fused with the fixed-point CIC deposit of Eq. (9)-(10)
//               and the (species, cell) histogram for the sort.
//   k_scatter4  counting-sort scatter A -> B by (species, cell).
//
// Both move four consecutive particles per thread with 128-bit loads issued
// before any of them is used, so that each warp keeps 512 B per array in
// flight: the kernels are bound by HBM latency and bandwidth, not by the
// arithmetic.  Slot arrays are padded to a multiple of four.
//
// Compiled with -fmad=false: every float operation is rounded on its own, in
// the order written, as in the reference formulas of the method.
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

// cell -> (iz, ir) without an integer division: float estimate, then fix by one
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

template <bool RZ, bool FIELD>
__global__ void __launch_bounds__(256) k_push4(Particles A, const float2* __restrict__ E, long long* rho_e,
                                               long long* rho_h, uint32_t* count, DevState* st, KParams P,
                                               PushConsts pc) {
    const uint32_t n = (uint32_t)st->n_slots;
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
        bool moved_any = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t i = 4u * g + (uint32_t)q;
            uint32_t key = (gv && i < n) ? lane_of(K, q) : DEAD;
            float pz = lane_of(Z, q), pr = lane_of(R, q);
            float vz = lane_of(VZ, q), vr = lane_of(VR, q), vt = lane_of(VT, q);
            ko[q] = lane_of(K, q);
            zo[q] = pz;
            ro[q] = pr;
            vzo[q] = vz;
            vro[q] = vr;
            vto[q] = vt;
            const bool live = key != DEAD;
            const int sp = (int)key_species(key);
            uint32_t cell = key_cell(key);
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
                    key = DEAD;
                    ko[q] = DEAD;
                    const double v2 = (double)vz * vz + (double)vr * vr + (double)vt * vt;
                    const double ke = P.weight * (0.5 * pick5(P.masses, sp) * v2);
                    atomicAdd(&st->ctr[C_ABS + electrode * NSP + sp], 1ull);
                    atomicAdd(&st->absorbed_energy[electrode], ke);
                    const double qw = (double)charge_of(sp) * 1.602176634e-19 * P.weight;
                    if (electrode == 1) atomicAdd(&st->anode_charge_step, qw);
                    if (electrode == 0) atomicAdd(&st->charge_cathode, qw);
                } else {
                    cell = (uint32_t)niz * (uint32_t)P.nr + (uint32_t)nir;
                    key = make_key((uint32_t)sp, cell);
                    ko[q] = key;
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
            const int zq = charge_of(sp);
            const bool dep = move && keep && zq != 0;
            // electrons and heavies deposit into separate grids (heavies are
            // held between their sub-cycled pushes)
            warp_deposit(rho_e, P, key, iz, ir, pz, pr, zq, dep && sp == SP_E);
            warp_deposit(rho_h, P, key, iz, ir, pz, pr, zq, dep && sp != SP_E);
            warp_count(count, (uint32_t)sp * P.ncell + cell, keep);
        }
        if (gv && moved_any) {
            key4[g] = make_uint4(ko[0], ko[1], ko[2], ko[3]);
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

// Counting-sort scatter.  All seven arrays of four particles are loaded
// first; then per particle: its bin offset and, for each group of lanes with
// the same bin, one atomic that reserves the group's slots (the bin counter
// counts back down to zero, ready for the next histogram).
__global__ void __launch_bounds__(256) k_scatter4(Particles A, Particles B, const uint32_t* __restrict__ off,
                                                  uint32_t* count, DevState* st, KParams P) {
    const uint32_t n = (uint32_t)st->n_slots;
    const uint32_t nv = (n + 3u) >> 2;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    const unsigned lt = lanemask_lt();
    for (uint32_t g0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); g0 < nv; g0 += stride) {
        const uint32_t g = g0 + lane;
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
        uint32_t bin[4], grp[4], base[4], old[4];
        bool lv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t key = (gv && 4u * g + (uint32_t)q < n) ? lane_of(K, q) : DEAD;
            lv[q] = key != DEAD;
            bin[q] = lv[q] ? key_species(key) * P.ncell + key_cell(key) : 0u;
            base[q] = lv[q] ? off[bin[q]] : 0u;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const unsigned m = __ballot_sync(FULL_MASK, lv[q]);
            grp[q] = lv[q] ? __match_any_sync(m, bin[q]) : 0u;
            old[q] = 0;
            if (lv[q] && lane == __ffs(grp[q]) - 1) old[q] = atomicSub(&count[bin[q]], (uint32_t)__popc(grp[q]));
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!lv[q]) continue;
            const uint32_t o = __shfl_sync(grp[q], old[q], __ffs(grp[q]) - 1);
            const uint32_t slot = base[q] + o - (uint32_t)__popc(grp[q]) + (uint32_t)__popc(grp[q] & lt);
            B.key[slot] = lane_of(K, q);
            B.pz[slot] = lane_of(Z, q);
            B.pr[slot] = lane_of(R, q);
            B.vz[slot] = lane_of(VZ, q);
            B.vr[slot] = lane_of(VR, q);
            B.vt[slot] = lane_of(VT, q);
            B.id[slot] = lane_of(ID, q);
        }
    }
}

void launch_push(const Particles& A, const float2* E, long long* rho_e, long long* rho_h, uint32_t* count,
                 DevState* st, const KParams& P, const PushConsts& pc, int grid, cudaStream_t s) {
    const bool rz = P.geom == 0, field = P.field_on != 0;
    if (rz && field) k_push4<true, true><<<grid, 256, 0, s>>>(A, E, rho_e, rho_h, count, st, P, pc);
    else if (rz) k_push4<true, false><<<grid, 256, 0, s>>>(A, E, rho_e, rho_h, count, st, P, pc);
    else if (field) k_push4<false, true><<<grid, 256, 0, s>>>(A, E, rho_e, rho_h, count, st, P, pc);
    else k_push4<false, false><<<grid, 256, 0, s>>>(A, E, rho_e, rho_h, count, st, P, pc);
}

void launch_scatter(const Particles& A, const Particles& B, const uint32_t* off, uint32_t* count, DevState* st,
                    const KParams& P, int grid, cudaStream_t s) {
    k_scatter4<<<grid, 256, 0, s>>>(A, B, off, count, st, P);
}

}  // namespace pd
