// pd_stream.cu -- the particle-streaming kernels of the step.
//
//   k_push4       Newton push (Sec. 2.1) with the field gathered by the CIC
//                 weights of Eq. (10), r-z rotation or periodic wrap,
//                 absorbing walls, fused with the fixed-point CIC deposit of
//                 Eq. (9)-(10) and the bookkeeping of the cell sort.
//   k_bins        per heavy bin: new count, overflow check, closing of the
//                 holes the push left (short bins; long ones are queued for
//                 k_compact_big, a warp per bin).
//   k_borrow      a full heavy bin takes free slots of the next bin.
//   k_relayout_*  a new slot layout of the heavy bins when one ran out of
//                 slots.
//   k_ebins, k_insert, k_insert_dense
//                 the electron bins packed after the heavy ones, and every
//                 mover into its new bin.
//
// The sort exploits that a step moves few heavy particles out of their
// (species, cell) bin.  Every heavy bin owns a fixed range of slots with
// slack after its live particles.  A heavy particle that stays in its bin
// ("stayer") stays in its slot: the push writes it back in place (on the
// steps that move no heavies it is not touched at all).  A heavy particle
// that leaves its bin or changed species in the collisions is a mover: the
// push copies it into the mover buffer at its slot's index and marks the slot
// it vacates.  The holes of each bin are then filled by the bin's last live
// particles, and the movers take the slots after the live ones of their new
// bin, one atomic cursor per bin.  A bin that receives more movers than it
// has free slots borrows the free slots of the next bin when that one is not
// full as of the counts; beyond that the heavy bins get a new layout (a
// counting sort into the second buffer, copied back), with slack sized from
// each bin's traffic since the previous layout.  Every kernel of the
// re-layout returns at once on the steps that need none, so the step's
// launch sequence is fixed (CUDA graphs).
//
// Electrons cross a cell in a few steps, so they are all movers: they sit in
// bins packed after the heavy region, and every step the push copies each
// one (with the particles created since the last sort, in the tail) into the
// mover buffer; a scan of the movers-in counts gives the electron bins'
// starts, and each mover takes its slot by the bin's atomic cursor.  The
// order inside a bin is not canonical (ascending id is found where it
// matters, in the collisions).
//
// The push moves four consecutive particles per thread with 128-bit loads
// issued before use.  Sorted input means the four usually share a cell, so
// counts and deposited charge are merged over runs of equal keys inside the
// thread (no warp-wide collectives on the common path), and the push
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

// the key of a particle converted by the last collisions (not a free slot)
__device__ __forceinline__ bool flagged(uint32_t k) { return k != DEAD && (k & KEY_FLAG); }

// mv: slots vacated in their heavy bin this step (bit per slot); mm: slots
// whose particle is in the mover buffer M; out_cnt / in_cnt: particles
// leaving / entering each bin.  Every electron is a mover (the electron bins
// are rebuilt each step), and so is every particle of the tail.
template <bool RZ, bool FIELD, bool MULTI>
__global__ void __launch_bounds__(256, (RZ || FIELD) ? 3 : 4) k_push4(Particles A, const float2* __restrict__ E, long long* rho_e,
                                               long long* rho_h, uint32_t* out_cnt, uint32_t* in_cnt,
                                               uint32_t* mv, uint32_t* mm, Particles M, DevState* st, KParams P) {
    __shared__ RunInfo s_runs[MULTI ? MAX_RUNS_SMEM : 1];
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    if (MULTI) {
        for (int r = threadIdx.x; r < P.nruns; r += blockDim.x) s_runs[r] = P.runs[r];
        __syncthreads();
    }
    const uint32_t n = (uint32_t)st->n_slots;
    const uint32_t n_sorted = (uint32_t)st->e_base;      // slots of the heavy bins; the electron bins follow
    if (blockIdx.x == 0 && threadIdx.x == 0) st->e_from = n_sorted;
    const uint32_t nv = (n + 3u) >> 2;
    const uint32_t stride = gridDim.x * blockDim.x;
    const int geom = RZ ? 0 : 1;
    uint4* key4 = reinterpret_cast<uint4*>(A.key);
    float4* pz4 = reinterpret_cast<float4*>(A.pz);
    float4* pr4 = reinterpret_cast<float4*>(A.pr);
    float4* vz4 = reinterpret_cast<float4*>(A.vz);
    float4* vr4 = reinterpret_cast<float4*>(A.vr);
    float4* vt4 = reinterpret_cast<float4*>(A.vt);
    const uint4 dead4 = make_uint4(DEAD, DEAD, DEAD, DEAD);
    uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    uint4 Kn = g < nv ? key4[g] : dead4;     // the keys of the thread's next group, loaded one group ahead
    for (; g - threadIdx.x % 32u < nv; g += stride) {
        const bool gv = g < nv;
        const uint4 K = Kn;
        Kn = g + stride < nv ? key4[g + stride] : dead4;
        float4 Z = make_float4(0, 0, 0, 0), R4 = Z, VZ = Z, VR = Z, VT = Z;
        // groups of four free slots (the bins' slack) read only their keys;
        // heavies move on heavy steps only, so on the other steps a group of
        // the heavy bins needs work only where the last collisions converted
        // a particle (it changes bin)
        const bool need = gv && (K.x & K.y & K.z & K.w) != DEAD &&
                          (P.heavy_step || 4u * g + 4u > n_sorted || flagged(K.x) || flagged(K.y) || flagged(K.z) ||
                           flagged(K.w));
        if (!__any_sync(FULL_MASK, need)) continue;
        if (need) {
            Z = pz4[g];
            R4 = pr4[g];
            VZ = vz4[g];
            VR = vr4[g];
            if (RZ) VT = vt4[g];
        }
        if constexpr (!RZ && !FIELD && !MULTI) {
            // Neutral copper staying in its cell.  On a heavy step, when every
            // live particle of the warp's groups is a neutral copper atom of
            // the heavy bins (its key carries no conversion) whose new
            // position stays inside its cell, the step below reduces to the new
            // positions written back in place: it keeps the key, the bin and
            // the velocity, deposits nothing, and its position update is the
            // same float operations (z - floor(z) is z + 0 when floor(z) is
            // zero, which also turns -0 into +0 as the subtraction does).
            if (P.heavy_step) {
                const float dtz = P.run0.dtz[1], dtr = P.run0.dtr[1];
                bool fast = true, anyl = false;
                float zs[4], rs[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t i = 4u * g + (uint32_t)q;
                    const uint32_t key_in = (gv && i < n) ? lane_of(K, q) : DEAD;
                    const float pz = lane_of(Z, q), pr = lane_of(R4, q);
                    const float z = pz + lane_of(VZ, q) * dtz;
                    const float rr = pr + lane_of(VR, q) * dtr;
                    const bool live = key_in != DEAD;
                    const bool stay = z >= 0.0f && z < 1.0f && rr >= 0.0f && rr < 1.0f;
                    fast = fast && (!live || ((key_in >> 24) == (uint32_t)SP_CU && i < n_sorted && stay));
                    anyl = anyl || live;
                    zs[q] = live ? z + 0.0f : pz;
                    rs[q] = live ? rr + 0.0f : pr;
                }
                if (__all_sync(FULL_MASK, fast || !need)) {
                    if (need && anyl) {
                        pz4[g] = make_float4(zs[0], zs[1], zs[2], zs[3]);
                        pr4[g] = make_float4(rs[0], rs[1], rs[2], rs[3]);
                    }
                    continue;
                }
            }
        }
        uint32_t key[4], newbin[4], oldbin[4];
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
            bool fin;        // the new position is finite (a fault upstream makes it NaN or infinite)
            if (RZ) {
                const float x = ((float)ir + pr) + vr * dtr;
                const float y = vt * dtr;
                const float rr = sqrtf(x * x + y * y);
                fin = isfinite(z) && isfinite(rr);
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
                // a finite step stays within one period, so the indices are in range
                fin = (unsigned)niz < (unsigned)RI.nz && (unsigned)nir < (unsigned)RI.nr;
            }
            // a non-finite position (a fault upstream) would index outside the
            // grid: the particle is dropped and the error flagged
            const bool bad = move && !fin;
            if (bad) set_error(st, ERR_NONFINITE);
            const bool absorbed = move && (out || bad);
            const bool kp = live && !absorbed;
            const uint32_t gcell =
                move ? RI.cell_base + (uint32_t)niz * (uint32_t)RI.nr + (uint32_t)nir : gcell_in;
            const uint32_t k = kp ? make_key((uint32_t)sp, gcell) : DEAD;
            const uint32_t nb = kp ? (uint32_t)sp * P.ncell + gcell : NOBIN;
            const bool mvq = in_sorted && nb != oldbin[q];
            const bool inq = kp && (!in_sorted || nb != oldbin[q]);
            const bool mk = move && kp;
            key[q] = k;
            newbin[q] = nb;
            mover[q] = mvq;
            inmv[q] = inq;
            absd[q] = absorbed && !bad;                   // (ledgers and impacts of finite particles only)
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
            // 16: the particle moved and keeps its slot (written back); a
            // mover's slot is refilled by the sort, an absorbed one's too
            flags |= (absorbed ? 1u : 0u) | (mvq ? 2u : 0u) | (inq ? 4u : 0u) | (dep[q] ? 8u : 0u) |
                     ((mk && !inq) ? 16u : 0u);
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
            uint32_t nib = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (len[q]) atomicAdd(&in_cnt[newbin[q]], len[q]);
                nib |= (inmv[q] ? 1u : 0u) << q;
            }
            if (nib) {
                // the group's new state into the mover buffer (lanes that are
                // not movers are never read); the Cartesian push does not
                // load v_theta, which it leaves unchanged
                reinterpret_cast<uint4*>(M.key)[g] = make_uint4(key[0], key[1], key[2], key[3]);
                reinterpret_cast<float4*>(M.pz)[g] = make_float4(zo[0], zo[1], zo[2], zo[3]);
                reinterpret_cast<float4*>(M.pr)[g] = make_float4(ro[0], ro[1], ro[2], ro[3]);
                reinterpret_cast<float4*>(M.vz)[g] = make_float4(vzo[0], vzo[1], vzo[2], vzo[3]);
                reinterpret_cast<float4*>(M.vr)[g] = make_float4(vro[0], vro[1], vro[2], vro[3]);
                reinterpret_cast<float4*>(M.vt)[g] = RZ ? make_float4(vto[0], vto[1], vto[2], vto[3]) : vt4[g];
                reinterpret_cast<uint4*>(M.id)[g] = reinterpret_cast<const uint4*>(A.id)[g];
                atomicOr(&mm[g >> 3], nib << (4u * (g & 7u)));
            }
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
        // write back the particles that moved and keep their slot (keys do not
        // change there)
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

// ---------------------------------------------------------------------
// sort: holes, insertions, re-layout
// ---------------------------------------------------------------------
// a failed consistency check of the sort: the sticky bounds error and, for
// diagnosis, which check (a bit per check site)
__device__ __forceinline__ void sort_fault(DevState* st, uint32_t where) {
    set_error(st, ERR_BOUNDS);
    atomicOr(&st->sort_fault, where);
}

__device__ __forceinline__ bool bit_of(const uint32_t* __restrict__ w, uint32_t i) { return (w[i >> 5] >> (i & 31u)) & 1u; }

// first slot in [from, to) whose bit is `want` (to if none)
__device__ __forceinline__ uint32_t next_bit(const uint32_t* __restrict__ w, uint32_t from, uint32_t to, bool want) {
    while (from < to) {
        uint32_t x = w[from >> 5];
        if (!want) x = ~x;
        x &= ~0u << (from & 31u);
        if (x) return min(to, (from & ~31u) + (uint32_t)(__ffs((int)x) - 1));
        from = (from & ~31u) + 32u;
    }
    return to;
}

__device__ __forceinline__ void move_slot(Particles& A, uint32_t from, uint32_t to) {
    A.key[to] = A.key[from];
    A.pz[to] = A.pz[from];
    A.pr[to] = A.pr[from];
    A.vz[to] = A.vz[from];
    A.vr[to] = A.vr[from];
    A.vt[to] = A.vt[from];
    A.id[to] = A.id[from];
}

// Bins of up to this many particles close their holes in k_bins (one
// thread); longer ones are queued for k_compact_big (one warp).
constexpr uint32_t COMPACT_THREAD_MAX = 96;

// Per heavy bin (b0 = the first) with traffic this step: the count after the movers out (c0) and in
// (cnt), the overflow check against the bin's slots, and the holes of
// [start, start + c) closed by moving the live particles of
// [start + c0, start + c) into them; that range then reads DEAD.
__global__ void __launch_bounds__(256) k_bins(Particles A, const uint32_t* __restrict__ off, uint32_t* cnt,
                                              uint32_t* out_cnt, const uint32_t* __restrict__ in_cnt,
                                              const uint32_t* __restrict__ mv, uint32_t* act, int* net, uint4* bigq,
                                              uint32_t bigq_cap, uint32_t* ovq, uint32_t* ovbits, uint32_t b0,
                                              uint32_t nbins, DevState* st) {
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    long long dlive = 0;
    for (uint32_t b = b0 + blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        const uint32_t o = out_cnt[b], in = in_cnt[b];
        if ((o | in) == 0u) continue;
        const uint32_t c = cnt[b];
        if (o > c) {                                   // inconsistent bookkeeping: report, move nothing
            sort_fault(st, 1u);
            continue;
        }
        const uint32_t c0 = c - o, cf = c0 + in;
        const uint32_t start = off[b];
        cnt[b] = cf;
        act[b] += o + in;
        net[b] += (int)in - (int)o;
        dlive += (long long)in - (long long)o;
        if (cf > off[b + 1] - start) {             // full: borrow from the next bin, else a new layout
            atomicOr(&ovbits[b >> 5], 1u << (b & 31u));
            const uint32_t q = atomicAdd(&st->n_ovf, 1u);
            if (q < OVQ_CAP) ovq[q] = b;
            else st->relayout = 1u;
        }
        if (o == 0u) continue;
        out_cnt[b] = 0u;
        if (c > COMPACT_THREAD_MAX) {
            const uint32_t q = atomicAdd(&st->n_bigc, 1u);
            if (q < bigq_cap) bigq[q] = make_uint4(b, start, c, c0);
            else sort_fault(st, 2u);
            continue;
        }
        const uint32_t end0 = start + c0, end = start + c;
        uint32_t h = start, j = end0;
        for (;;) {
            h = next_bit(mv, h, end0, true);           // a hole below the new count
            if (h >= end0) break;
            j = next_bit(mv, j, end, false);           // a live particle above it
            if (j >= end) {                            // cannot happen with consistent counts
                sort_fault(st, 4u);
                break;
            }
            move_slot(A, j, h);
            ++h;
            ++j;
        }
        for (uint32_t k = end0; k < end; ++k) A.key[k] = DEAD;
    }
    // the change of the live count, one atomic per block
    __shared__ long long s_d[8];
    const long long w = warp_sum_ll(dlive);
    if ((threadIdx.x & 31u) == 0u) s_d[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_d[k];
        if (t) atomicAdd(&st->n_live, (unsigned long long)t);
    }
}

// The same closing of holes for the queued long bins, a warp per bin: each
// round takes the holes of the next 32 slots below the new count and pairs
// them, in order, with the next live particles above it.
__global__ void __launch_bounds__(256) k_compact_big(Particles A, const uint32_t* __restrict__ mv,
                                                     const uint4* __restrict__ bigq, uint32_t bigq_cap,
                                                     DevState* st) {
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    __shared__ uint32_t s_h[8][32];
    const int lane = threadIdx.x & 31;
    uint32_t* sh = s_h[threadIdx.x >> 5];
    const uint32_t nq = min(st->n_bigc, bigq_cap);
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq; q += (gridDim.x * blockDim.x) >> 5) {
        const uint4 e = bigq[q];
        const uint32_t start = e.y, end = start + e.z, end0 = start + e.w;
        uint32_t hc = start, lc = end0;
        bool bad = false;
        while (hc < end0 && !bad) {
            const uint32_t sh_slot = hc + (uint32_t)lane;
            const bool hole = sh_slot < end0 && bit_of(mv, sh_slot);
            const uint32_t Hm = __ballot_sync(FULL_MASK, hole);
            hc += 32u;
            const uint32_t nh = (uint32_t)__popc(Hm);
            if (nh == 0u) continue;
            if (hole) sh[__popc(Hm & lt)] = sh_slot;
            __syncwarp();
            uint32_t got = 0;
            while (got < nh) {
                if (lc >= end) {                       // fewer live particles than holes: inconsistent counts
                    bad = true;
                    break;
                }
                const uint32_t sl = lc + (uint32_t)lane;
                const bool live = sl < end && !bit_of(mv, sl);
                const uint32_t Lm = __ballot_sync(FULL_MASK, live);
                const uint32_t nl = (uint32_t)__popc(Lm);
                const uint32_t take = min(nl, nh - got);
                const uint32_t lr = (uint32_t)__popc(Lm & lt);
                if (live && lr < take) move_slot(A, sl, sh[got + lr]);
                if (take == nl) {
                    lc += 32u;
                } else {
                    // past the take-th live slot of this chunk
                    uint32_t m = Lm;
                    for (uint32_t k = 1; k < take; ++k) m &= m - 1u;
                    lc += (uint32_t)__ffs((int)m);
                }
                got += take;
            }
            __syncwarp();
        }
        __syncwarp();
        if (bad) {
            if (lane == 0) sort_fault(st, 8u);
            continue;
        }
        for (uint32_t k = end0 + (uint32_t)lane; k < end; k += 32u) A.key[k] = DEAD;
    }
}

// A bin that outgrew its slots this step takes free slots from the next
// bin (same memory order: the next cell's bin of the species, or the first
// bin of the next species): the next bin's start moves up by `take` slots
// and the first of its live particles move to just after the others, at
// most `take` moves.  The next bin must not be full itself (its bit in
// ovbits, set before any borrowing) and must fit with `take` fewer slots; it
// lends half of what it can spare beyond the need.  A bin lends only to the
// bin before it and a full bin never lends: the offsets and slots a thread
// reads and writes are touched by no other thread.  Without such a
// neighbour the bins are laid out anew.
__global__ void __launch_bounds__(256) k_borrow(Particles A, uint32_t* off, const uint32_t* __restrict__ cnt,
                                                const uint32_t* __restrict__ in_cnt, const uint32_t* __restrict__ ovq,
                                                const uint32_t* __restrict__ ovbits, uint32_t nbins, DevState* st) {
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    const uint32_t nq = st->n_ovf;
    if (nq > OVQ_CAP) return;                        // (the re-layout is already set)
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const uint32_t b = ovq[q], l = b + 1u;
        const uint32_t need = cnt[b] - (off[b + 1] - off[b]);
        if (l >= nbins || bit_of(ovbits, l)) {
            st->relayout = 1u;
            continue;
        }
        const uint32_t lo = off[l], lcap = off[l + 1] - lo, lf = cnt[l];
        if (lf > lcap || lcap - lf < need) {
            st->relayout = 1u;
            continue;
        }
        const uint32_t take = need + (lcap - lf - need) / 2u;
        const uint32_t c0 = lf - in_cnt[l];              // the lender's live particles before its movers
        const uint32_t m = min(take, c0);
        const uint32_t nlo = lo + take;
        for (uint32_t j = 0; j < m; ++j) {
            const uint32_t src = lo + j, dst = nlo + c0 - m + j;
            move_slot(A, src, dst);
            A.key[src] = DEAD;
        }
        off[l] = nlo;
    }
}

// mover record i of M into slot s of D
__device__ __forceinline__ void put(Particles& D, uint32_t s, const Particles& M, uint32_t i) {
    D.key[s] = M.key[i];
    D.pz[s] = M.pz[i];
    D.pr[s] = M.pr[i];
    D.vz[s] = M.vz[i];
    D.vr[s] = M.vr[i];
    D.vt[s] = M.vt[i];
    D.id[s] = M.id[i];
}

// bin of a mover record's key (nbins if the key is not a particle's)
__device__ __forceinline__ uint32_t mover_bin(uint32_t k, uint32_t ncell, uint32_t nbins) {
    if (k == DEAD || key_cell(k) >= ncell) return nbins;
    const uint32_t b = key_species(k) * ncell + key_cell(k);
    return b < nbins ? b : nbins;
}

// The sparse movers of 128 slots (one uint4 of the mask) into bins laid out
// by `off`, after the live ones (cnt: the count after the insertions,
// in_cnt: the bin's cursor, back to zero when all its movers are in).
// heavy_only: electrons are left in the mask for the electron pass.
__device__ __forceinline__ void insert128(Particles& D, const Particles& M, uint32_t* mm, uint32_t g,
                                          const uint32_t* __restrict__ off, const uint32_t* __restrict__ cnt,
                                          uint32_t* in_cnt, uint32_t ncell, uint32_t nbins, uint32_t nslots,
                                          bool heavy_only, DevState* st) {
    const uint4 w = reinterpret_cast<uint4*>(mm)[g];
    if ((w.x | w.y | w.z | w.w) == 0u) return;
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    uint32_t keep[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t bits = ws[k];
        while (bits) {
            const uint32_t bit = (uint32_t)(__ffs((int)bits) - 1);
            bits &= bits - 1u;
            const uint32_t i = 128u * g + 32u * (uint32_t)k + bit;
            const uint32_t key = M.key[i];
            if (heavy_only && key != DEAD && key_species(key) == SP_E) {
                keep[k] |= 1u << bit;
                continue;
            }
            const uint32_t bin = mover_bin(key, ncell, nbins);
            if (bin >= nbins) {
                sort_fault(st, 128u);
                continue;
            }
            const uint32_t left = atomicSub(&in_cnt[bin], 1u);
            const uint32_t s = off[bin] + cnt[bin] - left;
            if (left == 0u || s >= off[bin] + cnt[bin] || s >= nslots) {   // inconsistent: report, never write out of range
                sort_fault(st, 16u);
                continue;
            }
            put(D, s, M, i);
        }
    }
    reinterpret_cast<uint4*>(mm)[g] = make_uint4(keep[0], keep[1], keep[2], keep[3]);
}

// heavy movers of the heavy bins' slots, in whole chunks of 128 below
// e_from (sparse: a thread per chunk)
__global__ void __launch_bounds__(256) k_insert(Particles A, Particles M, uint32_t* mm,
                                                const uint32_t* __restrict__ off, const uint32_t* __restrict__ cnt,
                                                uint32_t* in_cnt, uint32_t ncell, uint32_t nbins, uint32_t nslots,
                                                DevState* st) {
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    const uint32_t ng = (uint32_t)(st->e_from >> 7);
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
        insert128(A, M, mm, g, off, cnt, in_cnt, ncell, nbins, nslots, false, st);
}

// The movers from the first chunk of 128 that k_insert leaves (it ends below
// e_from) to the end of the tail: the electron bins and the tail (dense:
// every electron moves), and the last heavy slots before them.  A warp per
// chunk of 128 slots, as four rows of 32 consecutive slots, lane l taking
// slot l of each row: a row's records load in coalesced 128-byte lines, and
// the movers of a row that share a bin (consecutive slots of one old cell,
// mostly) take consecutive slots of it in lane order, so that each store
// writes runs of neighbouring words instead of one word per 32-byte sector.
// One atomic per bin and row claims the slots; the four rows' claims are
// issued before any result is used, beside the loads of the bins' ends.
__global__ void __launch_bounds__(256) k_insert_dense(Particles A, Particles M, const uint32_t* __restrict__ mm,
                                                      const uint32_t* __restrict__ off,
                                                      const uint32_t* __restrict__ cnt, uint32_t* in_cnt,
                                                      uint32_t ncell, uint32_t nbins, uint32_t nslots, DevState* st) {
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    const uint32_t n = (uint32_t)st->n_slots;
    const uint32_t c0 = (uint32_t)(st->e_from >> 7), c1 = (n + 127u) >> 7;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t c = c0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); c < c1; c += nwarps) {
        uint32_t K[4], ID[4];
        float Z[4], R[4], VZ[4], VR[4], VT[4];
        uint32_t bin[4], end[4], left[4];
        unsigned peers[4];
        bool ok[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t i = 128u * c + 32u * (uint32_t)q + lane;   // < 128 c1 <= the slot arrays' length
            const bool on = ((mm[4u * c + (uint32_t)q] >> lane) & 1u) && i < n;
            K[q] = M.key[i];
            Z[q] = M.pz[i];
            R[q] = M.pr[i];
            VZ[q] = M.vz[i];
            VR[q] = M.vr[i];
            VT[q] = M.vt[i];
            ID[q] = M.id[i];
            bin[q] = on ? mover_bin(K[q], ncell, nbins) : nbins;
            if (on && bin[q] >= nbins) sort_fault(st, 128u);
            ok[q] = on && bin[q] < nbins;
            end[q] = ok[q] ? off[bin[q]] + cnt[bin[q]] : 0u;
            peers[q] = __match_any_sync(FULL_MASK, ok[q] ? bin[q] : 0xFFFFFFFFu);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t leader = (uint32_t)(__ffs((int)peers[q]) - 1);
            left[q] = (ok[q] && lane == leader) ? atomicSub(&in_cnt[bin[q]], (uint32_t)__popc(peers[q])) : 0u;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t leader = (uint32_t)(__ffs((int)peers[q]) - 1);
            const uint32_t lq = __shfl_sync(FULL_MASK, left[q], (int)leader);
            if (!ok[q]) continue;
            const uint32_t rank = (uint32_t)__popc(peers[q] & ((1u << lane) - 1u));
            const uint32_t sl = end[q] - lq + rank;
            if (lq < (uint32_t)__popc(peers[q]) || sl >= end[q] || sl >= nslots) {
                sort_fault(st, 256u);
                continue;
            }
            A.key[sl] = K[q];
            A.pz[sl] = Z[q];
            A.pr[sl] = R[q];
            A.vz[sl] = VZ[q];
            A.vr[sl] = VR[q];
            A.vt[sl] = VT[q];
            A.id[sl] = ID[q];
        }
    }
}

// The electron bins, packed after the heavy bins: count = the electrons
// moving in (every electron), start = e_base + exclusive prefix of the counts
// (scanned into pre[]); the tail starts after them.
__global__ void __launch_bounds__(256) k_ebins(uint32_t* off, uint32_t* cnt, const uint32_t* __restrict__ in_cnt,
                                               const uint32_t* __restrict__ pre, uint32_t ncell, uint32_t nslots,
                                               DevState* st) {
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    const uint32_t eb = (uint32_t)st->e_base;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        off[c] = eb + pre[c];
        cnt[c] = in_cnt[c];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->n_e = pre[ncell];
        st->tail_base = (unsigned long long)eb + pre[ncell];
        if (st->tail_base > nslots) set_error(st, ERR_CAPACITY);   // the inserts then write nothing past the slots
    }
}

// ---- re-layout (only on steps where a bin overflowed) ----------------
// Slack of a bin: room for a random walk of its movers in and out and for
// its drift over H steps, SLACK_SIGMAS standard deviations (a layout holds
// about a million bins):
//     slack = 3 + ceil(SLACK_SIGMAS sqrt(lambda H) + drift H)
// (the constant covers the heavier tail of small counts: a bin's arrivals
// are Poisson).
// lambda, a bin's traffic per step, is the larger of its own since the
// previous layout and its species' traffic per particle times the larger of
// its count and the species' mean count per bin (a short interval sees no
// traffic in many bins that do have it, and particles flow into a bin from
// its neighbours, empty or not).  H is the largest horizon up to
// SLACK_HORIZON_MAX steps whose slack fits in the slots beyond the configured
// capacity, so that the layout lasts about H steps.  Without history (the
// first layout) the slack is a sixteenth of the count and two.
constexpr float SLACK_HORIZON_MAX = 100.0f;
constexpr float SLACK_SIGMAS = 5.3f;

// per species: particles and traffic over the bins
__global__ void __launch_bounds__(256) k_relayout_stats(const uint32_t* __restrict__ cnt,
                                                        const uint32_t* __restrict__ act, uint32_t nbins,
                                                        uint32_t ncell, int nsp, DevState* st) {
    if (!st->relayout || st->error) return;
    unsigned long long c_[NSP], a_[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) c_[k] = a_[k] = 0ull;
    for (uint32_t b = ncell + blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        const uint32_t sp = b / ncell, c = cnt[b], a = act[b];
#pragma unroll
        for (int k = 0; k < NSP; ++k) {
            c_[k] += sp == (uint32_t)k ? c : 0u;
            a_[k] += sp == (uint32_t)k ? a : 0u;
        }
    }
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
        if (k >= nsp) break;
        const unsigned long long wc = warp_sum_ull(c_[k]), wa = warp_sum_ull(a_[k]);
        if ((threadIdx.x & 31u) == 0u) {
            if (wc) atomicAdd(&st->sp_cnt[k], wc);
            if (wa) atomicAdd(&st->sp_act[k], wa);
        }
    }
}

// a bin's traffic per step (lambda) and drift per step
__device__ __forceinline__ void bin_traffic(uint32_t b, uint32_t c, uint32_t a, int nt, uint32_t since, uint32_t ncell,
                                            const float* s_rate, const float* s_mean, float& lam, float& drift) {
    const uint32_t sp = b / ncell;
    const float own = (float)a / (float)since;
    lam = fmaxf(own, s_rate[sp] * fmaxf((float)c, s_mean[sp]));
    drift = fmaxf((float)nt, 0.0f) / (float)since;
}

__device__ __forceinline__ void species_rates(const DevState* st, uint32_t since, uint32_t ncell, float* s_rate,
                                              float* s_mean) {
    if (threadIdx.x < NSP) {
        const unsigned long long c = st->sp_cnt[threadIdx.x];
        s_rate[threadIdx.x] = (since > 0u && c > 0ull)
                                  ? (float)((double)st->sp_act[threadIdx.x] / ((double)c * (double)since))
                                  : 0.0f;
        s_mean[threadIdx.x] = (float)((double)c / (double)ncell);
    }
    __syncthreads();
}

// sums over the heavy bins of the count, of SLACK_SIGMAS sqrt(lambda) and of the drift
__global__ void __launch_bounds__(256) k_relayout_want(const uint32_t* __restrict__ cnt,
                                                       const uint32_t* __restrict__ act, const int* __restrict__ net,
                                                       uint32_t nbins, uint32_t ncell, DevState* st) {
    if (!st->relayout || st->error) return;
    const uint32_t since = st->since;
    __shared__ float s_rate[NSP], s_mean[NSP];
    species_rates(st, since, ncell, s_rate, s_mean);
    unsigned long long sc = 0;
    double s1 = 0.0, s2 = 0.0;
    for (uint32_t b = ncell + blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        const uint32_t c = cnt[b];
        sc += c;
        if (since == 0u) continue;
        float lam, drift;
        bin_traffic(b, c, act[b], net[b], since, ncell, s_rate, s_mean, lam, drift);
        s1 += (double)(SLACK_SIGMAS * sqrtf(lam));
        s2 += (double)drift;
    }
    __shared__ unsigned long long s_c[8];
    __shared__ double s_1[8], s_2[8];
    sc = warp_sum_ull(sc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(FULL_MASK, s1, o);
        s2 += __shfl_xor_sync(FULL_MASK, s2, o);
    }
    if ((threadIdx.x & 31u) == 0u) {
        s_c[threadIdx.x >> 5] = sc;
        s_1[threadIdx.x >> 5] = s1;
        s_2[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tc = 0;
        double t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            tc += s_c[k];
            t1 += s_1[k];
            t2 += s_2[k];
        }
        atomicAdd(&st->sum_cnt, tc);
        atomicAdd(&st->sum_s1, t1);
        atomicAdd(&st->sum_s2, t2);
    }
}

// heavy bin capacities: count plus slack over the horizon that fits the
// slots beyond the configured capacity (the electron bins get none: they are
// packed after the heavy bins every step); history cleared
__global__ void __launch_bounds__(256) k_relayout_caps(const uint32_t* __restrict__ cnt, uint32_t* cap,
                                                       uint32_t* act, int* net, uint32_t nbins, uint32_t nbins_pad,
                                                       uint32_t ncell, DevState* st, KParams P) {
    if (!st->relayout || st->error) return;
    const uint32_t since = st->since;
    __shared__ float s_rate[NSP], s_mean[NSP];
    species_rates(st, since, ncell, s_rate, s_mean);
    // room for the slack: the slots beyond the capacity (or beyond the
    // particles, if more), less four slots per bin (the three added and the
    // rounding up)
    const unsigned long long used = max(st->sum_cnt + st->n_e + 1024ull, P.user_capacity) + 4ull * nbins;
    const double room = P.capacity > used ? (double)(P.capacity - used) : 0.0;
    // largest H <= SLACK_HORIZON_MAX with s1 sqrt(H) + s2 H <= room
    const double s1 = st->sum_s1, s2 = st->sum_s2;
    double x;
    if (s2 > 0.0) x = (-s1 + sqrt(s1 * s1 + 4.0 * s2 * room)) / (2.0 * s2);
    else x = s1 > 0.0 ? room / s1 : 1e30;
    const float H = (float)fmin((double)SLACK_HORIZON_MAX, x * x), sqH = sqrtf(H);
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins_pad; b += gridDim.x * blockDim.x) {
        if (b >= nbins || b < ncell) {
            cap[b] = 0u;
            continue;
        }
        const uint32_t c = cnt[b];
        uint32_t w;
        if (since == 0u) {
            w = 2u + (c >> 4);
        } else {
            float lam, drift;
            bin_traffic(b, c, act[b], net[b], since, ncell, s_rate, s_mean, lam, drift);
            w = 3u + (uint32_t)ceilf(SLACK_SIGMAS * sqrtf(lam) * sqH + drift * H);
        }
        cap[b] = c + w;
        act[b] = 0u;
        net[b] = 0;
    }
}

// B's keys over the new bins: DEAD (slack slots stay so)
__global__ void __launch_bounds__(256) k_relayout_clear(uint32_t* key, const uint32_t* __restrict__ off2,
                                                        uint32_t nbins, DevState* st) {
    if (!st->relayout || st->error) return;
    const uint32_t nv = (off2[nbins] + 3u) >> 2;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x)
        reinterpret_cast<uint4*>(key)[v] = make_uint4(DEAD, DEAD, DEAD, DEAD);
}

// B := the heavy particles in the new layout off2: the live particles of
// each heavy bin (its first cnt - in slots after the closing of holes) keep
// their order, the heavy movers follow them.  Clears the heavy movers' bits
// of the mover mask (the electrons are inserted after the electron bins are
// laid out).  A warp per 128 slots, lane l taking slot l of each row of 32:
// the loads and the stores of a row are runs of consecutive words (a bin
// keeps its order and moves by one offset).  in_place: B is A itself, which
// holds only while no particle sits in a bin (the first layout after the
// loads, every particle a mover).
__global__ void __launch_bounds__(256) k_relayout_scatter(Particles A, Particles B, Particles M,
                                                          uint32_t* mm, const uint32_t* __restrict__ off,
                                                          const uint32_t* __restrict__ off2,
                                                          const uint32_t* __restrict__ cnt, uint32_t* in_cnt,
                                                          uint32_t nbins, DevState* st, KParams P, bool in_place) {
    if (!st->relayout || st->error) return;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t tb = (uint32_t)st->e_from, nch = (tb + 127u) >> 7;
    if (in_place && tb != 0u) {        // B is A: only valid while no particle sits in a bin
        sort_fault(st, 512u);
        return;
    }
    for (uint32_t c = tid >> 5; c < nch; c += stride >> 5) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // (the last chunk may reach into the electron bins: they are movers)
            const uint32_t i = 128u * c + 32u * (uint32_t)q + lane;
            if (i >= tb) continue;
            const uint32_t k = A.key[i];
            if (k == DEAD) continue;
            const uint32_t b = key_species(k) * P.ncell + key_cell(k);
            if (key_cell(k) >= P.ncell || b >= nbins || i < off[b] || i - off[b] >= cnt[b]) {
                sort_fault(st, 64u);             // not a particle of its bin: never write out of range
                continue;
            }
            const uint32_t s = off2[b] + (i - off[b]);
            B.key[s] = k;
            B.pz[s] = A.pz[i];
            B.pr[s] = A.pr[i];
            B.vz[s] = A.vz[i];
            B.vr[s] = A.vr[i];
            B.vt[s] = A.vt[i];
            B.id[s] = A.id[i];
        }
    }
    // The heavy movers, a warp per 128 slots of the mover mask (lane l takes
    // slot l of each row of 32).  After a load every particle is a mover, so
    // the rows are dense: the movers of a row bound for one bin claim their
    // slots with one atomic, and the records' loads of the four rows are in
    // flight together.  Electrons stay in the mask for the electron pass.
    const uint32_t ng = (uint32_t)((st->n_slots + 127ull) >> 7);
    const uint32_t nslots = (uint32_t)P.capacity;
    for (uint32_t g = tid >> 5; g < ng; g += stride >> 5) {
        const uint4 w = reinterpret_cast<const uint4*>(mm)[g];
        if ((w.x | w.y | w.z | w.w) == 0u) continue;          // the same chunk in every lane
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
        uint32_t K[4], bin[4], end[4], left[4];
        unsigned peers[4];
        bool ok[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t i = 128u * g + 32u * (uint32_t)q + lane;    // < 128 ng <= the slot arrays' length
            const bool on = (ws[q] >> lane) & 1u;
            K[q] = on ? M.key[i] : DEAD;
            const bool elec = on && K[q] != DEAD && key_species(K[q]) == SP_E;
            const bool heavy = on && !elec;
            bin[q] = heavy ? mover_bin(K[q], P.ncell, nbins) : nbins;
            if (heavy && bin[q] >= nbins) sort_fault(st, 128u);
            ok[q] = heavy && bin[q] < nbins;
            end[q] = ok[q] ? off2[bin[q]] + cnt[bin[q]] : 0u;
            peers[q] = __match_any_sync(FULL_MASK, ok[q] ? bin[q] : 0xFFFFFFFFu);
            const unsigned keep = __ballot_sync(FULL_MASK, elec);
            if (lane == 0u) mm[4u * g + (uint32_t)q] = keep;
        }
        float Z[4], R[4], VZ[4], VR[4], VT[4];
        uint32_t ID[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t i = 128u * g + 32u * (uint32_t)q + lane;
            const uint32_t leader = (uint32_t)(__ffs((int)peers[q]) - 1);
            left[q] = (ok[q] && lane == leader) ? atomicSub(&in_cnt[bin[q]], (uint32_t)__popc(peers[q])) : 0u;
            Z[q] = ok[q] ? M.pz[i] : 0.0f;
            R[q] = ok[q] ? M.pr[i] : 0.0f;
            VZ[q] = ok[q] ? M.vz[i] : 0.0f;
            VR[q] = ok[q] ? M.vr[i] : 0.0f;
            VT[q] = ok[q] ? M.vt[i] : 0.0f;
            ID[q] = ok[q] ? M.id[i] : 0u;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t leader = (uint32_t)(__ffs((int)peers[q]) - 1);
            const uint32_t lq = __shfl_sync(FULL_MASK, left[q], (int)leader);
            if (!ok[q]) continue;
            const uint32_t rank = (uint32_t)__popc(peers[q] & ((1u << lane) - 1u));
            const uint32_t s = end[q] - lq + rank;
            if (lq < (uint32_t)__popc(peers[q]) || s >= end[q] || s >= nslots) {   // inconsistent: never write out of range
                sort_fault(st, 16u);
                continue;
            }
            B.key[s] = K[q];
            B.pz[s] = Z[q];
            B.pr[s] = R[q];
            B.vz[s] = VZ[q];
            B.vr[s] = VR[q];
            B.vt[s] = VT[q];
            B.id[s] = ID[q];
        }
    }
}

// A := B over the new heavy bins (groups of four slack slots copy only
// their keys), off := off2; the electron bins start after them.  in_place:
// the re-layout was written into A itself (nothing to copy)
__global__ void __launch_bounds__(256) k_relayout_copy(Particles A, Particles B, uint32_t* off,
                                                       const uint32_t* __restrict__ off2, uint32_t nbins,
                                                       uint32_t nbins_pad, DevState* st, bool in_place) {
    if (!st->relayout || st->error) return;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t end = off2[nbins], nv = in_place ? 0u : (end + 3u) >> 2;
    for (uint32_t v = tid; v < nv; v += stride) {
        uint4 K = reinterpret_cast<const uint4*>(B.key)[v];
        if (4u * v + 4u > end) {       // the last group: slots past the bins read DEAD
            if (4u * v + 1u > end) K.y = DEAD;
            if (4u * v + 2u > end) K.z = DEAD;
            if (4u * v + 3u > end) K.w = DEAD;
        }
        reinterpret_cast<uint4*>(A.key)[v] = K;
        if ((K.x & K.y & K.z & K.w) == DEAD) continue;
        reinterpret_cast<float4*>(A.pz)[v] = reinterpret_cast<const float4*>(B.pz)[v];
        reinterpret_cast<float4*>(A.pr)[v] = reinterpret_cast<const float4*>(B.pr)[v];
        reinterpret_cast<float4*>(A.vz)[v] = reinterpret_cast<const float4*>(B.vz)[v];
        reinterpret_cast<float4*>(A.vr)[v] = reinterpret_cast<const float4*>(B.vr)[v];
        reinterpret_cast<float4*>(A.vt)[v] = reinterpret_cast<const float4*>(B.vt)[v];
        reinterpret_cast<uint4*>(A.id)[v] = reinterpret_cast<const uint4*>(B.id)[v];
    }
    for (uint32_t b = tid; b <= nbins_pad; b += stride) off[b] = off2[b];
}

// after the copy: the re-layout is done
__global__ void k_relayout_done(const uint32_t* __restrict__ off, uint32_t nbins, DevState* st) {
    if (!st->relayout || st->error) return;
    st->e_base = off[nbins];
    st->relayout = 0u;
    st->since = 0u;
    st->n_relayout += 1u;
    st->sum_cnt = 0ull;
    st->sum_s1 = st->sum_s2 = 0.0;
    for (int k = 0; k < NSP; ++k) st->sp_cnt[k] = st->sp_act[k] = 0ull;
}

void launch_push(const Particles& A, const float2* E, long long* rho_e, long long* rho_h, uint32_t* out_cnt,
                 uint32_t* in_cnt, uint32_t* mv, uint32_t* mm, const Particles& M, DevState* st, const KParams& P,
                 int grid, cudaStream_t s) {
    const bool rz = P.geom == 0, field = P.field_on != 0;
#define PD_PUSH_ARGS A, E, rho_e, rho_h, out_cnt, in_cnt, mv, mm, M, st, P
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

void launch_sort(const SortArgs& a, DevState* st, const KParams& P, int sms, cudaStream_t s) {
    // one thread per heavy bin: the work of a thread is a chain of dependent
    // loads, which many threads in flight hide
    const uint32_t gb = (a.nbins - P.ncell + 255u) / 256u;
    cudaMemsetAsync(a.ovbits, 0, (size_t)(a.nbins / 32u + 1u) * 4u, s);
    k_bins<<<gb, 256, 0, s>>>(a.A, a.off, a.cnt, a.out_cnt, a.in_cnt, a.mv, a.act, a.net, a.bigq, a.bigq_cap, a.ovq,
                              a.ovbits, P.ncell, a.nbins, st);
    k_compact_big<<<sms * 4, 256, 0, s>>>(a.A, a.mv, a.bigq, a.bigq_cap, st);
    k_borrow<<<(OVQ_CAP + 255u) / 256u, 256, 0, s>>>(a.A, a.off, a.cnt, a.in_cnt, a.ovq, a.ovbits, a.nbins, st);
}

void launch_relayout(const SortArgs& a, DevState* st, const KParams& P, int grid_bins, int grid_slots,
                     cudaStream_t s, bool first) {
    // each kernel returns at once unless a bin overflowed.  The first layout
    // (no particle in any bin yet: every loaded particle is a mover) is
    // written straight into A, and nothing is copied back.
    const Particles& D = first ? a.A : a.B;
    k_relayout_stats<<<grid_bins, 256, 0, s>>>(a.cnt, a.act, a.nbins, P.ncell, P.nsp, st);
    k_relayout_want<<<grid_bins, 256, 0, s>>>(a.cnt, a.act, a.net, a.nbins, P.ncell, st);
    k_relayout_caps<<<grid_bins, 256, 0, s>>>(a.cnt, a.cap, a.act, a.net, a.nbins, a.nbins_pad, P.ncell, st, P);
    launch_scan(a.cap, a.off2, a.partial, a.nbins_pad, s, &st->relayout);
    k_relayout_clear<<<grid_slots, 256, 0, s>>>(D.key, a.off2, a.nbins, st);
    k_relayout_scatter<<<grid_slots, 256, 0, s>>>(a.A, D, a.M, a.mm, a.off, a.off2, a.cnt, a.in_cnt, a.nbins, st,
                                                  P, first);
    k_relayout_copy<<<grid_slots, 256, 0, s>>>(a.A, D, a.off, a.off2, a.nbins, a.nbins_pad, st, first);
    k_relayout_done<<<1, 1, 0, s>>>(a.off, a.nbins, st);
}

void launch_insert(const SortArgs& a, DevState* st, const KParams& P, int grid_dense, cudaStream_t s) {
    // the electron bins: counts scanned (into off2, free after a re-layout), laid out after the heavy bins
    launch_scan(a.in_cnt, a.off2, a.partial, a.ncell_pad, s);
    k_ebins<<<(P.ncell + 255u) / 256u, 256, 0, s>>>(a.off, a.cnt, a.in_cnt, a.off2, P.ncell, (uint32_t)a.slots, st);
    // heavy movers (a thread per 128 slots of the heavy bins), then the electrons and the tail
    const uint32_t gs = (uint32_t)((a.slots / 128u + 255u) / 256u);
    k_insert<<<gs, 256, 0, s>>>(a.A, a.M, a.mm, a.off, a.cnt, a.in_cnt, P.ncell, a.nbins, (uint32_t)a.slots, st);
    k_insert_dense<<<grid_dense, 256, 0, s>>>(a.A, a.M, a.mm, a.off, a.cnt, a.in_cnt, P.ncell, a.nbins,
                                              (uint32_t)a.slots, st);
}

}  // namespace pd
