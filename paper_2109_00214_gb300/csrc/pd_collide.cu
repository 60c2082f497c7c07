// pd_collide.cu -- DSMC electron-impact collisions and cathode injection.
//
// Collisions (Sec. 2.1 Eq. (4)-(7), Sec. 2.2 Eq. (11)-(20)) in no-time-counter
// form, per cell and pair class k in {(e, Cu), (e, Cu+)}:
//   k_ncand    N_cand = floor(N_e N_t c_k(r) + R), c_k = W (sigma g)_max dt_coll / V_cell,
//              one thread per cell; cells with candidates go to an active list.
//              Lists of more than RANK_WARP_MAX ids that active cells use
//              are queued for k_rank_tables.
//   k_rank_tables  rank tables of the queued lists, one block per list.
//   k_collide  one warp per active cell.  Candidate m draws from the stream
//              (cell, step, k<<28 | m): the electron and target ranks (in
//              ascending-id order inside the cell), the acceptance number and
//              the channel number.  Lane 0 applies the kinematics.  Spawned electrons go to the slots
//              reserved for the cell at n_alive + 2 * (candidates of the
//              cells before it); unused reserved slots are marked dead.
//   k_finalize slot / id bookkeeping and the RC circuit update.
// Compiled with -fmad=false (decision arithmetic is rounded op by op).
#include "pd_internal.cuh"
#include "pd_kernels.h"

namespace pd {

constexpr unsigned FULL = 0xFFFFFFFFu;

struct V3 {
    float x, y, z;
};

// isotropic unit vector, Marsaglia (1972)
__device__ V3 iso_dir(Stream& st, uint32_t& fb) {
    for (int a = 0; a < 64; ++a) {
        const float u1 = 2.0f * st.u01() - 1.0f;
        const float u2 = 2.0f * st.u01() - 1.0f;
        const float s = u1 * u1 + u2 * u2;
        if (s < 1.0f) {
            const float q = 2.0f * sqrtf(1.0f - s);
            return V3{u1 * q, u2 * q, 1.0f - 2.0f * s};
        }
    }
    ++fb;
    return V3{0.0f, 0.0f, 1.0f};
}

// uniform azimuth (cos, sin) from a point of the unit disc
__device__ void azimuth(Stream& st, float& c, float& s, uint32_t& fb) {
    for (int a = 0; a < 64; ++a) {
        const float u1 = 2.0f * st.u01() - 1.0f;
        const float u2 = 2.0f * st.u01() - 1.0f;
        const float q = u1 * u1 + u2 * u2;
        if (q < 1.0f && q > 0.0f) {
            const float r = sqrtf(q);
            c = u1 / r;
            s = u2 / r;
            return;
        }
    }
    ++fb;
    c = 1.0f;
    s = 0.0f;
}

// Eq. (6): |u'|^2 = |u|^2 - 2 E_th / m_r (kth); Eq. (7) isotropic direction;
// Eq. (5): v1 += (u' - u) m_r/m1, v2 -= (u' - u) m_r/m2.
__device__ bool binary_scatter(Stream& st, V3& v1, V3& v2, float kth, float a1, float a2, uint32_t& fb) {
    const V3 u{v1.x - v2.x, v1.y - v2.y, v1.z - v2.z};
    const float g2 = (u.x * u.x + u.y * u.y) + u.z * u.z;
    const float up2 = g2 - kth;
    if (up2 < 0.0f) return false;
    const float gp = sqrtf(up2);
    const V3 n = iso_dir(st, fb);
    const V3 du{gp * n.x - u.x, gp * n.y - u.y, gp * n.z - u.z};
    v1.x = v1.x + du.x * a1;
    v1.y = v1.y + du.y * a1;
    v1.z = v1.z + du.z * a1;
    v2.x = v2.x - du.x * a2;
    v2.y = v2.y - du.y * a2;
    v2.z = v2.z - du.z * a2;
    return true;
}

// Eq. (15)-(20): v5 = cos(chi) |v| R^T(theta, phi) (sin chi cos psi,
// sin chi sin psi, cos chi); v6 = v - v5; theta, phi from the components of v.
__device__ void rectangle_split(Stream& st, const V3& v, V3& v5, V3& v6, int mode, uint32_t& fb) {
    float cchi = st.u01();
    if (mode == 1) cchi = sqrtf(cchi);
    const float schi = sqrtf(1.0f - cchi * cchi);
    float cpsi, spsi;
    azimuth(st, cpsi, spsi, fb);
    const float vperp2 = v.x * v.x + v.y * v.y;
    const float vmag2 = vperp2 + v.z * v.z;
    const float vmag = sqrtf(vmag2), vperp = sqrtf(vperp2);
    V3 w5{0.0f, 0.0f, 0.0f};
    if (vmag > 0.0f) {
        const float ct = v.z / vmag, sth = vperp / vmag;
        float cp = 1.0f, sp = 0.0f;
        if (vperp > 0.0f) {
            cp = v.x / vperp;
            sp = v.y / vperp;
        }
        const float a = cchi * vmag;
        const float w1 = a * (schi * cpsi), w2 = a * (schi * spsi), w3 = a * cchi;
        w5.x = (w1 * (ct * cp) - w2 * sp) + w3 * (sth * cp);
        w5.y = (w1 * (ct * sp) + w2 * cp) + w3 * (sth * sp);
        w5.z = w3 * ct - w1 * sth;
    }
    v5 = w5;
    v6 = V3{v.x - w5.x, v.y - w5.y, v.z - w5.z};
}

// single-particle fixed-point CIC deposit of zq at (local cell, pz, pr) of run RI
__device__ void deposit1(long long* rho, const RunInfo& RI, int geom, uint32_t lcell, float pz, float pr, int zq) {
    const int iz = (int)(lcell / (uint32_t)RI.nr);
    const int ir = (int)(lcell - (uint32_t)iz * (uint32_t)RI.nr);
    const uint32_t wz = __float2uint_rn(pz * 65536.0f);
    const uint32_t wr = __float2uint_rn(pr * 65536.0f);
    const long long az = 65536 - (long long)wz, ar = 65536 - (long long)wr;
    atomicAdd((unsigned long long*)&rho[node_of(RI, geom, iz, ir)], (unsigned long long)(zq * az * ar));
    atomicAdd((unsigned long long*)&rho[node_of(RI, geom, iz + 1, ir)], (unsigned long long)(zq * (long long)wz * ar));
    atomicAdd((unsigned long long*)&rho[node_of(RI, geom, iz, ir + 1)], (unsigned long long)(zq * az * (long long)wr));
    atomicAdd((unsigned long long*)&rho[node_of(RI, geom, iz + 1, ir + 1)],
              (unsigned long long)(zq * (long long)wz * (long long)wr));
}

// Ranks inside a cell.  The candidate draws give ranks in ascending-id order;
// the sorted slots hold a cell's particles in an order that depends on the
// scatter's atomics, so each list the candidates use is mapped rank ->
// position by one of:
//   * ids already ascending with the position (rank = position);
//   * up to 64 ids: a rank table by comparisons (the rank of an id is the
//     number of smaller ids in the list);
//   * up to 32 * RC ids with lookups that cost less than a table: a radix
//     select over the ids held in registers, per lookup;
//   * longer lists with at most SELECT_LOOKUPS lookups: a select per lookup
//     over the list in global memory (select8);
//   * otherwise a rank table, position of the r-th smallest id at table[r],
//     from a stable LSD radix sort of (id, position) pairs by 8-bit digits:
//     by the cell's warp in its shared memory for the register-cached lists
//     (up to RANK_WARP_MAX = 32 * RC ids), by a block of k_rank_tables
//     (before k_collide) for longer lists, in shared memory up to
//     RANK_BLOCK_MAX ids and in the scratch buffers above that.
// The table of the list at slots [b, b + n) is written to table[b, b + n).

// Register-cached id list of one cell and species: element lane + 32 k in
// ids[k], for lists of up to 32 * RC ids (one coalesced load per cell).
constexpr int RC = 8;
constexpr uint32_t RANK_BLOCK_MAX = 12288;      // longest list the large kernel sorts in shared memory
constexpr int RT_THREADS = 1024;                // threads of a large-kernel block
constexpr int RT_MID_THREADS = 256;             // threads of a mid-size-kernel block
constexpr int RT_MID_BLOCKS_PER_SM = 5;
constexpr uint32_t SENTINEL = 0xFFFFFFFFu;

struct IdList {
    uint32_t ids[RC];
    const uint32_t* table;           // rank -> position, or null
    const uint32_t* base;            // the ids in global memory (select8)
    uint32_t* cnt;                   // the warp's 256 shared counters (select8)
    uint32_t n;
    int top;                         // highest set bit of any id (0 if none)
    bool cached;
    bool sorted;                     // ids ascend with the position: rank = position
    bool sel8;                       // a long list with few lookups: select8 per lookup
};

// lookups up to which a list longer than 32 * RC ids is searched per lookup
// (select8) instead of being sorted into a rank table: a select costs a few
// sweeps of the list by one warp, a table a few sweeps by a whole block
constexpr uint32_t SELECT_LOOKUPS = 4;

// The lanes of the warp whose 8-bit digit d equals this lane's (v: the
// lane holds a digit at all; lanes without one group with none), from nine
// ballots (a warp multisplit).
__device__ __forceinline__ unsigned digit_peers(uint32_t d, bool v) {
    unsigned peers = __ballot_sync(FULL, v);
    peers = v ? peers : ~peers;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const unsigned bb = __ballot_sync(FULL, bit);
        peers &= bit ? bb : ~bb;
    }
    return peers;
}

// Position of the rank-th smallest of the n (unique) ids at ids[0, n) by
// one warp: passes over windows of 8 bits from bit `top` (every id is below
// 2^(top + 1)) down, each counting, in the warp's 256 shared counters, the
// ids that share the bits found so far; SENTINEL if rank >= n.  The first
// window is the top 8 bits, so that its digits spread over the counters
// (windows aligned to bit 0 would leave the first pass one or two digits:
// every id's atomic on the same counters); the last window holds the bits
// that remain.  Each lane keeps eight loads in flight.
__device__ uint32_t select8(const uint32_t* __restrict__ ids, uint32_t n, uint32_t rank, int top, uint32_t* cnt,
                            int lane) {
    uint32_t prefix = 0, want = rank;
    for (int lo = top - 7;; lo -= 8) {
        const int sh = lo > 0 ? lo : 0;
        const int width = lo >= 0 ? 8 : 8 + lo;        // bits of this window
        const uint32_t dm = (1u << width) - 1u;
        const uint32_t hm = sh + width >= 32 ? 0u : (0xFFFFFFFFu << (sh + width));
#pragma unroll
        for (int k = 0; k < 8; ++k) cnt[lane * 8 + k] = 0u;
        __syncwarp();
        for (uint32_t q0 = 0; q0 < n; q0 += 256) {
            uint32_t x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t q = q0 + 32u * u + (uint32_t)lane;
                x[u] = q < n ? ids[q] : 0u;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t q = q0 + 32u * u + (uint32_t)lane;
                if (q < n && (x[u] & hm) == prefix) atomicAdd(&cnt[(x[u] >> sh) & dm], 1u);
            }
        }
        __syncwarp();
        uint32_t c[8], sum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            c[k] = cnt[lane * 8 + k];
            sum += c[k];
        }
        uint32_t xs = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, xs, o);
            if (lane >= o) xs += y;
        }
        const uint32_t before = xs - sum;
        const bool mine = want >= before && want < xs;
        uint32_t d = 0, rest = 0, run = before;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (mine && want >= run && want < run + c[k]) {
                d = (uint32_t)(lane * 8 + k);
                rest = want - run;
            }
            run += c[k];
        }
        const unsigned b = __ballot_sync(FULL, mine);
        __syncwarp();
        if (!b) return SENTINEL;
        const int src = __ffs(b) - 1;
        d = __shfl_sync(FULL, d, src);
        want = __shfl_sync(FULL, rest, src);
        prefix |= d << sh;
        if (sh == 0) break;
    }
    uint32_t pos = SENTINEL;
    for (uint32_t q0 = 0; q0 < n; q0 += 256) {
        uint32_t x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t q = q0 + 32u * u + (uint32_t)lane;
            x[u] = q < n ? ids[q] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t q = q0 + 32u * u + (uint32_t)lane;
            if (q < n && x[u] == prefix && q < pos) pos = q;
        }
    }
    return __reduce_min_sync(FULL, pos);
}

// Scratch of the rank tables, arrays indexed by slot: two (key, value) pair
// buffers and the tables.  They are the sort's other buffer, unused between
// the scatter and the next step's scatter; a list at slots [b, b + n) uses
// [b, b + n) of each.
struct RankScratch {
    uint32_t *xk, *xv, *yk, *yv, *table;
};

// One stable counting pass of an LSD radix sort over the pairs [0, n) by the
// first nw warps of the group (one warp: BLOCK false; the whole block:
// BLOCK true, all threads calling): warp w takes the w-th run of `seg`
// pairs.  Keys come from sk, values from sv (null: the position itself);
// the pairs go to (dk, dv) ordered by the digit (key >> sh) & 255, pairs of
// equal digits keeping their order (dk null: values only).  Per 32 pairs,
// digit_peers groups equal digits; a group's members take consecutive
// places after the digit's running offset in lane order and the group's
// highest lane advances it.  cnt: 256 counters per warp; tot: 256 (BLOCK).
template <bool BLOCK>
__device__ void radix_pass(const uint32_t* sk, const uint32_t* sv, uint32_t* dk, uint32_t* dv, uint32_t n, int sh,
                           int nw, uint32_t* cnt, uint32_t* tot, uint32_t tid, int lane, int w) {
    const uint32_t seg = (n + 32u * nw - 1) / (32u * nw) * 32u;
    const uint32_t q0 = min(n, (uint32_t)w * seg), q1 = min(n, q0 + seg);
    uint32_t* c = cnt + (BLOCK ? w * 256 : 0);
#pragma unroll
    for (int k = 0; k < 8; ++k) c[lane * 8 + k] = 0u;
    __syncwarp();
    for (uint32_t g = q0; g < q1; g += 32) {
        const uint32_t q = g + lane;
        const uint32_t d = q < q1 ? (sk[q] >> sh) & 255u : 256u;
        const unsigned peers = digit_peers(d, q < q1);
        if (q < q1 && lane == 31 - __clz((int)peers)) c[d] += (uint32_t)__popc(peers);
        __syncwarp();
    }
    // offsets: digit-major over the warps
    if (BLOCK) {
        __syncthreads();
        if (tid < 256) {
            uint32_t run = 0;
            for (int v = 0; v < nw; ++v) {
                const uint32_t x = cnt[v * 256 + tid];
                cnt[v * 256 + tid] = run;
                run += x;
            }
            tot[tid] = run;
        }
        __syncthreads();
    }
    if (!BLOCK || w == 0) {
        uint32_t* t = BLOCK ? tot : c;
        uint32_t cc[8], sum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            cc[k] = t[lane * 8 + k];
            sum += cc[k];
        }
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        uint32_t run = x - sum;
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            t[lane * 8 + k] = run;
            run += cc[k];
        }
        __syncwarp();
    }
    if (BLOCK) {
        __syncthreads();
        if (tid < 256)
            for (int v = 0; v < nw; ++v) cnt[v * 256 + tid] += tot[tid];
        __syncthreads();
    }
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    for (uint32_t g = q0; g < q1; g += 32) {
        const uint32_t q = g + lane;
        const bool in = q < q1;
        const uint32_t key = in ? sk[q] : 0u, val = in ? (sv ? sv[q] : q) : 0u;
        const uint32_t d = in ? (key >> sh) & 255u : 256u;
        const unsigned peers = digit_peers(d, in);
        const uint32_t b = in ? c[d] : 0u;
        __syncwarp();
        if (in) {
            if (lane == 31 - __clz((int)peers)) c[d] = b + (uint32_t)__popc(peers);
            const uint32_t dst = b + (uint32_t)__popc(peers & lt);
            if (dk) dk[dst] = key;
            dv[dst] = val;
        }
        __syncwarp();
    }
    if (BLOCK) __syncthreads();
    else __syncwarp();
}

// Rank table of the n ids staged in xk (unique; highest set bit `top`):
// the digits up to `top`, passes alternating between (yk, yv) and (xk, xv),
// the last one writing the positions to table.
template <bool BLOCK>
__device__ void radix_table(uint32_t n, int top, uint32_t* xk, uint32_t* xv, uint32_t* yk, uint32_t* yv,
                            uint32_t* table, int nw, uint32_t* cnt, uint32_t* tot, uint32_t tid, int lane, int w) {
    const int passes = top / 8 + 1;
    const uint32_t *sk = xk, *sv = nullptr;
    for (int p = 0; p < passes; ++p) {
        const bool last = p + 1 == passes;
        uint32_t* dk = last ? nullptr : ((p & 1) ? xk : yk);
        uint32_t* dv = last ? table : ((p & 1) ? xv : yv);
        radix_pass<BLOCK>(sk, sv, dk, dv, n, 8 * p, nw, cnt, tot, tid, lane, w);
        sk = dk;
        sv = dv;
    }
}

// Rank tables of the lists that k_collide will use and k_ncand queued for
// this kernel (entries cell << 3 | species bin 0..6; *nq of them, at most
// max_q): one list per block at a time, NT threads, sorted in shared memory
// up to MAXN ids and in the scratch buffers above that.  A list already in
// ascending id order gets the identity.
template <int NT, uint32_t MAXN>
__global__ void __launch_bounds__(NT) k_rank_tables(const uint32_t* __restrict__ ids, RankScratch S,
                                                    const uint32_t* __restrict__ off, const uint32_t* __restrict__ cnt,
                                                    const uint32_t* __restrict__ q,
                                                    const uint32_t* nq, uint32_t max_q, uint32_t C,
                                                    const DevState* st) {
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    constexpr int NWARPS = NT / 32;
    extern __shared__ uint32_t s_buf[];                 // four arrays of MAXN
    __shared__ uint32_t s_cnt[NWARPS * 256];
    __shared__ uint32_t s_tot[256];
    __shared__ uint32_t s_or;
    const uint32_t nb = min(*nq, max_q);             // an overflow is flagged by k_ncand
    const uint32_t tid = threadIdx.x;
    const int lane = (int)(tid & 31u), w = (int)(tid >> 5);
    if (tid == 0) s_or = 0u;
    __syncthreads();
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const uint32_t e = q[b];
        const uint32_t bin = (e & 7u) * C + (e >> 3);
        const uint32_t slot0 = off[bin], n = cnt[bin];
        const uint32_t* base = ids + slot0;
        const bool in_smem = n <= MAXN;
        uint32_t* xk = in_smem ? s_buf : S.xk + slot0;
        uint32_t* xv = in_smem ? s_buf + MAXN : S.xv + slot0;
        uint32_t* yk = in_smem ? s_buf + 2 * MAXN : S.yk + slot0;
        uint32_t* yv = in_smem ? s_buf + 3 * MAXN : S.yv + slot0;
        uint32_t* table = S.table + slot0;
        uint32_t orv = 0;
        for (uint32_t k = tid; k < n; k += NT) {
            const uint32_t x = base[k];
            xk[k] = x;
            orv |= x;
        }
        orv = __reduce_or_sync(FULL, orv);
        if (lane == 0 && orv) atomicOr(&s_or, orv);
        __syncthreads();
        bool asc = true;
        for (uint32_t k = tid; k + 1 < n; k += NT)
            if (!(xk[k] < xk[k + 1])) asc = false;
        const uint32_t any = s_or;
        if (__syncthreads_and(asc)) {
            for (uint32_t r = tid; r < n; r += NT) table[r] = r;
        } else {
            const int top = any ? 31 - __clz((int)any) : 0;
            const int nw = (int)min((uint32_t)NWARPS, (n + 255u) / 256u);
            radix_table<true>(n, top, xk, xv, yk, yv, table, nw, s_cnt, s_tot, tid, lane, w);
        }
        if (tid == 0) s_or = 0u;
        __syncthreads();
    }
}

// ids of one cell and species at slots [slot0, slot0 + n); `lookups` rank
// selections will follow.  sbuf: the warp's four arrays of RANK_WARP_MAX and
// its 256 counters.
__device__ __forceinline__ void load_ids(IdList& L, const uint32_t* __restrict__ ids, uint32_t slot0, uint32_t n,
                                         uint32_t lookups, const RankScratch& S, uint32_t* sbuf, int lane,
                                         int id_top, bool want_table = false) {
    const uint32_t* base = ids + slot0;
    L.n = n;
    L.table = nullptr;
    L.base = base;
    L.cnt = sbuf + 4 * RANK_WARP_MAX;
    L.cached = n <= 32u * RC;
    L.sorted = false;
    L.sel8 = false;
    L.top = 0;
    if (!want_table && !L.cached && lookups <= SELECT_LOOKUPS) {
        L.sel8 = true;
        L.top = id_top;
        return;
    }
    if (!L.cached) {                 // table built by k_rank_tables
        L.table = S.table + slot0;
        return;
    }
    uint32_t* xk = sbuf;
    bool asc = true;
    uint32_t orv = 0;
    if (L.cached) {
#pragma unroll
        for (int k = 0; k < RC; ++k) {
            const uint32_t q = (uint32_t)lane + 32u * k;
            L.ids[k] = q < n ? base[q] : 0u;
            orv |= L.ids[k];
        }
#pragma unroll
        for (int k = 0; k < RC; ++k) {
            // element q + 1 is lane + 1 of the same row, or lane 0 of the next
            const uint32_t q = (uint32_t)lane + 32u * k;
            const uint32_t right = __shfl_down_sync(FULL, L.ids[k], 1);
            const uint32_t wrap = __shfl_sync(FULL, k + 1 < RC ? L.ids[k + 1 < RC ? k + 1 : k] : 0u, 0);
            const uint32_t next = lane == 31 ? wrap : right;
            if (q + 1 < n && !(L.ids[k] < next)) asc = false;
        }
        orv = __reduce_or_sync(FULL, orv);
        L.top = orv ? 31 - __clz((int)orv) : 0;
        L.sorted = __all_sync(FULL, asc);
        if (L.sorted) return;
        if (n <= 64u) {
            // a short list's table by comparison: the rank of an id is the
            // number of smaller ids (ids are unique), 32 exchanges per row
            uint32_t r0 = 0, r1 = 0;
            if (n <= 32u) {
#pragma unroll 8
                for (int j = 0; j < 32; ++j) {
                    const uint32_t a = __shfl_sync(FULL, L.ids[0], j);
                    r0 += ((uint32_t)j < n && a < L.ids[0]) ? 1u : 0u;
                }
            } else {
#pragma unroll 8
                for (int j = 0; j < 32; ++j) {
                    const uint32_t a = __shfl_sync(FULL, L.ids[0], j), b = __shfl_sync(FULL, L.ids[1], j);
                    const bool vb = 32u + (uint32_t)j < n;
                    r0 += (a < L.ids[0] ? 1u : 0u) + (vb && b < L.ids[0] ? 1u : 0u);
                    r1 += (a < L.ids[1] ? 1u : 0u) + (vb && b < L.ids[1] ? 1u : 0u);
                }
            }
            uint32_t* table = S.table + slot0;
            if ((uint32_t)lane < n) table[r0] = (uint32_t)lane;
            if (32u + (uint32_t)lane < n) table[r1] = 32u + (uint32_t)lane;
            __syncwarp();
            L.table = table;
            L.cached = false;
            return;
        }
        // a select sweeps the registers once per significant bit, per lookup
        // (about 48 instructions a bit); the table takes a radix pass per
        // 8-bit digit (about 96 plus 64 per 32 ids)
        const uint32_t sel_cost = lookups * (uint32_t)(L.top + 1) * 48u;
        const uint32_t tab_cost = (uint32_t)(L.top / 8 + 1) * (96u + ((n + 31u) / 32u) * 64u);
        if (!want_table && sel_cost <= tab_cost) return;
#pragma unroll
        for (int k = 0; k < RC; ++k) {
            const uint32_t q = (uint32_t)lane + 32u * k;
            if (q < n) xk[q] = L.ids[k];
        }
    }
    __syncwarp();
    uint32_t* table = S.table + slot0;
    radix_table<false>(n, L.top, xk, sbuf + RANK_WARP_MAX, sbuf + 2 * RANK_WARP_MAX, sbuf + 3 * RANK_WARP_MAX, table,
                       1, sbuf + 4 * RANK_WARP_MAX, nullptr, (uint32_t)lane, lane, 0);
    L.table = table;                 // ordered for the warp by radix_pass's final __syncwarp
    L.cached = false;
}

// position of the rank-th smallest id of the list
__device__ __forceinline__ uint32_t select_rank_list(const IdList& L, uint32_t rank, int lane) {
    if (L.sorted) return rank;
    if (L.table) return L.table[rank];
    if (L.sel8) return select8(L.base, L.n, rank, L.top, L.cnt, lane);
    // register-cached list: bitwise radix select
    uint32_t prefix = 0, want = rank;
    for (int bit = L.top; bit >= 0; --bit) {
        const uint32_t hm = bit == 31 ? 0u : (0xFFFFFFFFu << (bit + 1));
        uint32_t cnt = 0;
#pragma unroll
        for (int k = 0; k < RC; ++k) {
            const uint32_t q = (uint32_t)lane + 32u * k;
            cnt += (q < L.n && (L.ids[k] & hm) == prefix && !((L.ids[k] >> bit) & 1u)) ? 1u : 0u;
        }
        cnt = __reduce_add_sync(FULL, cnt);
        if (want >= cnt) {
            want -= cnt;
            prefix |= 1u << bit;
        }
    }
    uint32_t pos = SENTINEL;
#pragma unroll
    for (int k = 0; k < RC; ++k) {
        const uint32_t q = (uint32_t)lane + 32u * k;
        if (q < L.n && L.ids[k] == prefix) pos = q;
    }
    return __reduce_min_sync(FULL, pos);
}

// Heavy cells (a list the warp must sort or many candidates) go to the
// front of `active`, the others to its back, so that k_collide starts them
// first.
// EXT: any of the step-wise, heavy-pair or Coulomb extensions is on (the
// plain variant counts the classes (e, Cu) and (e, Cu+) only)
template <bool EXT>
__global__ void __launch_bounds__(256) k_ncand(const uint32_t* __restrict__ cnt, const float* __restrict__ ck,
                                               uint4* nc, uint4* nc2, uint32_t* cand, uint32_t* active, uint32_t* mid,
                                               uint32_t* big, DevState* st, KParams P) {
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    const uint32_t C = P.ncell;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    const bool heavy_pairs = EXT && P.heavy_coll && P.heavy_step;
    const bool q3 = EXT && P.charge_max >= 3, q4 = EXT && P.charge_max >= 4;
    for (uint32_t c0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); c0 < C; c0 += stride) {
        const uint32_t c = c0 + lane;
        // n[k]: candidates of class k (electron classes 0-4, heavy pairs 5, 6)
        uint32_t n[NCLS] = {0, 0, 0, 0, 0, 0, 0};
        uint32_t N[NSP] = {0, 0, 0, 0, 0, 0, 0};
        int r = -1;
        if (c < C) {
            // list lengths (Cu3+ and Cu4+ have bins with charge_max >= 3; Cu4+ is
            // drawn only by the Coulomb pairs)
#pragma unroll
            for (int sp = 0; sp < NSP; ++sp)
                if ((sp < 5 || q3) && (sp < 6 || P.coulomb)) N[sp] = cnt[sp * C + c];
            const uint32_t Nt[NECLS] = {N[SP_CU], N[SP_CUP], N[SP_CU2_SW], N[SP_CU2_DI], N[SP_CU3]};
            bool ecls = false;
            for (int k = 0; k < NECLS; ++k) ecls |= Nt[k] > 0;
            ecls = ecls && N[SP_E] > 0;
            const bool hcls = heavy_pairs && N[SP_CU] > 0;
            if (ecls || hcls) {
                r = run_of(P, c);
                const RunInfo& RI = P.runs[r];
                const uint32_t lc = c - RI.cell_base;
                const uint32_t j = lc % (uint32_t)RI.nr;
                // the cell's stream gives R_k to class k whether the class is on or not
                Stream s(lc, st->step, SID_NCAND, RI.seed, RI.run);
                float R[NCLS];
#pragma unroll
                for (int k = 0; k < NCLS; ++k) R[k] = s.u01();
                if (ecls) {
#pragma unroll
                    for (int k = 0; k < NECLS; ++k) {
                        if (k >= 2 && !q3) break;
                        if (k == 4 && !q4) break;
                        const float x = ((float)N[SP_E] * (float)Nt[k]) * ck[RI.ck_base + k * RI.nr + j] + R[k];
                        n[k] = (uint32_t)floorf(x);
                    }
                }
                if (hcls) {
                    // N_cu N_cu+ charge-exchange pairs, N_cu (N_cu - 1) / 2 Cu-Cu
                    // pairs (the 1/2 is in the row factor)
                    const uint32_t Ncu = N[SP_CU], Ni = N[SP_CUP];
                    const float x5 = ((float)Ncu * (float)Ni) * ck[RI.ck_base + 5 * RI.nr + j] + R[5];
                    const float x6 = ((float)Ncu * (float)(Ncu - 1u)) * ck[RI.ck_base + 6 * RI.nr + j] + R[6];
                    n[5] = (uint32_t)floorf(x5);
                    n[6] = Ncu >= 2 ? (uint32_t)floorf(x6) : 0u;
                }
            }
            nc[c] = make_uint4(n[0], n[1], n[5], n[6]);
            if (q3) nc2[c] = make_uint4(n[2], n[3], n[4], 0u);
            cand[c] = n[0] + n[1] + n[2] + n[3] + n[4];    // the electron classes reserve spawn slots
        }
        // heavy candidates join the run's candidate count here (the electron
        // classes' are summed from the spawn-slot scan)
        const uint32_t nh = n[5] + n[6];
        if (__any_sync(FULL, nh > 0)) {
            const int r0 = __shfl_sync(FULL, r, 0);
            if (__all_sync(FULL, nh == 0 || r == r0)) {
                const uint32_t t = __reduce_add_sync(FULL, nh);
                if (lane == 0) atomicAdd(&P.rs[r0].ctr[C_CAND], (unsigned long long)t);
            } else if (nh > 0) {
                atomicAdd(&P.rs[r].ctr[C_CAND], (unsigned long long)nh);
            }
        }
        // lookups of each species' list over the classes that draw from it;
        // the Coulomb pairs look up every electron and every ion of a cell
        // with electrons (k_collide counts the same)
        uint32_t look[NSP];
        look[SP_E] = n[0] + n[1] + n[2] + n[3] + n[4];
        look[SP_CU] = n[0] + n[5] + 2u * n[6];
        look[SP_CUP] = n[1] + n[5];
        look[SP_CU2_SW] = n[2];
        look[SP_CU2_DI] = n[3];
        look[SP_CU3] = n[4];
        look[SP_CU4] = 0;
        uint32_t ncoul = 0;          // Coulomb pairs of the cell (about)
        if (EXT && P.coulomb && N[SP_E] > 0) {
            look[SP_E] += N[SP_E];
            ncoul = N[SP_E] / 2u;
#pragma unroll
            for (int sp = SP_CUP; sp < NSP; ++sp) ncoul += N[sp] > 0 ? max(N[SP_E], N[sp]) : 0u;
        }
        // the ion lists: with electrons, or on heavy steps (ion pairs)
        if (EXT && P.coulomb && (N[SP_E] > 0 || P.heavy_step)) {
#pragma unroll
            for (int sp = SP_CUP; sp < NSP; ++sp) {
                look[sp] += N[sp];
                ncoul += P.heavy_step ? N[sp] : 0u;
            }
        }
        // k_collide takes the cells with DSMC candidates; k_coulomb visits the
        // others itself, but the rank tables it needs are queued here too
        const uint32_t ntot = n[0] + n[1] + n[2] + n[3] + n[4] + nh;
        const bool act = c < C && ntot > 0;
        const uint32_t RL = 32u * RC;
        bool long_list = false;
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp) long_list |= look[sp] > 0 && N[sp] > RL;
        const bool heavy = act && (ntot > 32u || long_list);
        unsigned lt;
        asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
        const unsigned mh = __ballot_sync(FULL, heavy), ml = __ballot_sync(FULL, act && !heavy);
        uint32_t bh = 0, bl = 0;
        if (mh && lane == __ffs(mh) - 1) bh = atomicAdd(&st->n_heavy, (uint32_t)__popc(mh));
        if (ml && lane == __ffs(ml) - 1) bl = atomicAdd(&st->n_light, (uint32_t)__popc(ml));
        if (mh) bh = __shfl_sync(FULL, bh, __ffs(mh) - 1);
        if (ml) bl = __shfl_sync(FULL, bl, __ffs(ml) - 1);
        if (heavy) active[bh + __popc(mh & lt)] = c;
        else if (act) active[C - 1u - (bl + __popc(ml & lt))] = c;
        if (act || (c < C && ncoul > 0)) {
            // the lists k_collide or k_coulomb will rank that need a block's
            // sort (long, with more lookups than select8 serves)
            for (uint32_t sp = 0; sp < (uint32_t)NSP; ++sp) {
                if (look[sp] == 0 || N[sp] <= RANK_WARP_MAX || look[sp] <= SELECT_LOOKUPS) continue;
                const bool large = N[sp] > RANK_MID_MAX;
                const uint32_t x = atomicAdd(large ? &st->n_big : &st->n_mid, 1u);
                if (x < rank_queue_max(P.capacity, large ? RANK_MID_MAX : RANK_WARP_MAX))
                    (large ? big : mid)[x] = (c << 3) | sp;
                else set_error(st, ERR_BOUNDS);
            }
        }
    }
}

struct CellCtx {
    uint32_t cell;                   // global cell
    const RunInfo* RI;
    int geom;
    unsigned long long slot0;        // first reserved spawn slot
    uint32_t nres;                   // reserved slots
    uint32_t id0;                    // id of the first reserved slot
    uint32_t s;                      // spawned so far
    uint32_t ev[NCH], nulls, consumed, thr, viol, fb;
    uint32_t coul_ee, coul_ei, coul_ii;   // Coulomb pair collisions applied
};

__device__ bool spawn_electron(Particles& A, CellCtx& cx, DevState* st, long long* rho_e, uint32_t gcell, float pz,
                               float pr, const V3& v) {
    if (cx.s >= cx.nres) {
        set_error(st, ERR_BOUNDS);
        return false;
    }
    const unsigned long long slot = cx.slot0 + cx.s;
    A.key[slot] = make_key(SP_E, gcell);
    A.pz[slot] = pz;
    A.pr[slot] = pr;
    A.vz[slot] = v.x;
    A.vr[slot] = v.y;
    A.vt[slot] = v.z;
    A.id[slot] = cx.id0 + cx.s;
    ++cx.s;
    deposit1(rho_e, *cx.RI, cx.geom, gcell - cx.RI->cell_base, pz, pr, -1);
    return true;
}

// lane-0 part of one candidate after the pair is chosen
// cross sections of a pair: running sums cum[] of the class's channels at
// the pair's relative energy, and sigma_T g
struct PairEval {
    float cum[4];
    float sg;
};

// pair classes: first channel and target species of class k (the electron
// classes draw an electron as the first particle, the heavy pairs a Cu)
__device__ __forceinline__ int class_ch0(int k) {
    return k == 0 ? CH_EL : k == 1 ? CH_SW : k <= 3 ? CH_S3 : k == 4 ? CH_S4 : k == 5 ? CH_CX : CH_NN;
}
__device__ __forceinline__ int class_target(int k) {
    return k == 0 ? SP_CU : k == 1 ? SP_CUP : k == 2 ? SP_CU2_SW : k == 3 ? SP_CU2_DI : k == 4 ? SP_CU3
         : k == 5 ? SP_CUP : SP_CU;
}

__device__ __forceinline__ PairEval evaluate_pair(int k, const V3& ve, const V3& vt, const float* __restrict__ xsE,
                                                  const float* __restrict__ xs, const CollConsts& cc) {
    PairEval e;
    const float ux = ve.x - vt.x, uy = ve.y - vt.y, uz = ve.z - vt.z;
    const float g2 = (ux * ux + uy * uy) + uz * uz;
    const float g = sqrtf(g2);
    const float eps = g2 * (k < NECLS ? cc.kmr : cc.kmr_h);
    const int ch0 = class_ch0(k);
    const int nch = k == 0 ? 4 : 1;
    float sT = 0.0f;
    for (int q = 0; q < 4; ++q) {
        if (q < nch) sT = sT + xs_lookup(xsE, xs + (ch0 + q) * XS_N, eps);
        e.cum[q] = sT;
    }
    e.sg = sT * g;
    return e;
}

// (tkey, ve, vt: the target's key and both velocities as they are now; ev:
// evaluate_pair of ve, vt)
// (accepted: the candidate is known to pass the target and acceptance
// tests, already counted by the caller)
__device__ void process_candidate(Particles& A, CellCtx& cx, Stream& rs, int k, uint32_t ie, uint32_t it,
                                  uint32_t tkey, V3 ve, V3 vt, const PairEval& ev, float Racc, float Rch,
                                  const float* __restrict__ xsE, const float* __restrict__ xs,
                                  const CollConsts& cc, DevState* st, long long* rho_e, long long* rho_h,
                                  bool accepted) {
    const int ts = class_target(k);
    if (!accepted && ((tkey & KEY_FLAG) || (int)key_species(tkey) != ts)) {   // target already ionized this step
        ++cx.consumed;
        return;
    }
    const int ch0 = class_ch0(k);
    const int nch = k == 0 ? 4 : 1;
    const float* cum = ev.cum;
    const float sT = cum[nch - 1];
    const float sg = ev.sg;
    if (!accepted) {
        if (sg > cc.sgmax[k]) ++cx.viol;
        if (!(Racc * cc.sgmax[k] < sg)) {
            ++cx.nulls;
            return;
        }
    }
    const float r = Rch * sT;
    int q = -1;
    for (int a = 0; a < nch; ++a)
        if (r < cum[a]) {
            q = a;
            break;
        }
    if (q < 0) {
        q = nch - 1;
        for (int a = nch - 1; a >= 0; --a)
            if (cum[a] > (a ? cum[a - 1] : 0.0f)) {
                q = a;
                break;
            }
    }
    const int ch = ch0 + q;
    if (ch == CH_EL || ch == CH_EXC) {
        if (!binary_scatter(rs, ve, vt, ch == CH_EL ? 0.0f : cc.kth[ch], cc.a_e, cc.a_t, cx.fb)) {
            ++cx.thr;
            return;
        }
        A.vz[ie] = ve.x; A.vr[ie] = ve.y; A.vt[ie] = ve.z;
        A.vz[it] = vt.x; A.vr[it] = vt.y; A.vt[it] = vt.z;
        ++cx.ev[ch];
        return;
    }
    // Stage 1, Eq. (12): e + A -> e1 + A*, losing the threshold energy
    if (!binary_scatter(rs, ve, vt, cc.kth[ch], cc.a_e, cc.a_t, cx.fb)) {
        ++cx.thr;
        return;
    }
    // Stage 2, Eq. (13): A* -> e2 + ion with the position and velocity of A*
    V3 e2 = vt;
    // Stage 3, Eq. (14): e1 + e2 elastic, equal masses
    binary_scatter(rs, ve, e2, 0.0f, 0.5f, 0.5f, cx.fb);
    const int new_sp = ch == CH_SI ? SP_CUP : ch == CH_SW ? SP_CU2_SW : ch == CH_DI ? SP_CU2_DI
                     : ch == CH_S3 ? SP_CU3 : SP_CU4;
    const int dq = charge_of(new_sp) - charge_of(ts);
    V3 keep = ve, e6{0.0f, 0.0f, 0.0f};
    if (ch == CH_DI) {
        // Stage 4, Eq. (15): e3 -> e5 + e6 (velocity rectangle)
        V3 e5;
        rectangle_split(rs, ve, e5, e6, cc.di_split_mode, cx.fb);
        keep = e5;
    }
    A.vz[ie] = keep.x; A.vr[ie] = keep.y; A.vt[ie] = keep.z;
    A.vz[it] = vt.x; A.vr[it] = vt.y; A.vt[it] = vt.z;
    const uint32_t tcell = key_cell(tkey);
    A.key[it] = converted_key((uint32_t)new_sp, (uint32_t)ts, tcell);
    const float tpz = A.pz[it], tpr = A.pr[it];
    deposit1(rho_h, *cx.RI, cx.geom, tcell - cx.RI->cell_base, tpz, tpr, dq);
    spawn_electron(A, cx, st, rho_e, tcell, tpz, tpr, e2);
    if (ch == CH_DI) spawn_electron(A, cx, st, rho_e, key_cell(A.key[ie]), A.pz[ie], A.pr[ie], e6);
    ++cx.ev[ch];
}

// a pair whose particles are no longer what its class draws: a target
// ionized earlier this step or, for the heavy classes, a Cu that was
__device__ __forceinline__ bool consumed_pair(int k, uint32_t akey, uint32_t tkey) {
    const int ts = class_target(k);
    const bool t_gone = (tkey & KEY_FLAG) || (int)key_species(tkey) != ts;
    if (k < NECLS) return t_gone;
    return t_gone || (akey & KEY_FLAG) || (int)key_species(akey) != SP_CU;
}

// lane-0 part of one heavy-pair candidate (classes 5 and 6: one channel
// each, nothing spawned), the counterpart of process_candidate.  Charge
// exchange Cu + Cu+ -> Cu+ + Cu moves the electron, not the atoms: each slot
// keeps its species and takes the other's velocity.  Cu + Cu is elastic and
// isotropic in the centre of mass, equal masses.
__device__ void process_heavy_pair(Particles& A, CellCtx& cx, Stream& rs, int k, uint32_t ia, uint32_t ib,
                                   uint32_t akey, uint32_t bkey, V3 va, V3 vb, const PairEval& ev, float Racc,
                                   const CollConsts& cc, bool accepted) {
    if (!accepted) {
        if (consumed_pair(k, akey, bkey)) {
            ++cx.consumed;
            return;
        }
        if (ev.sg > cc.sgmax[k]) ++cx.viol;
        if (!(Racc * cc.sgmax[k] < ev.sg)) {
            ++cx.nulls;
            return;
        }
    }
    if (k == 5) {
        A.vz[ia] = vb.x; A.vr[ia] = vb.y; A.vt[ia] = vb.z;
        A.vz[ib] = va.x; A.vr[ib] = va.y; A.vt[ib] = va.z;
        ++cx.ev[CH_CX];
        return;
    }
    binary_scatter(rs, va, vb, 0.0f, 0.5f, 0.5f, cx.fb);
    A.vz[ia] = va.x; A.vr[ia] = va.y; A.vt[ia] = va.z;
    A.vz[ib] = vb.x; A.vr[ib] = vb.y; A.vt[ib] = vb.z;
    ++cx.ev[CH_NN];
}

// ---------------------------------------------------------------------
// Coulomb collisions (listed by Sec. 2.3 without a method): the binary
// collision model of Takizuka and Abe (1977).  A pair with relative velocity
// u turns by theta, tan(theta / 2) = delta, delta = sqrt(Kn / u^3) Z with Z
// normal (here the Irwin-Hall sum of twelve uniforms), about a uniform
// azimuth; |u| is kept and the change is shared by the reduced mass.  Kn =
// (q_a q_b)^2 n_L lnL dt / (8 pi eps0^2 m_ab^2).  The float operations are
// those of the oracle's float build, in the same order.
//
// A pair's particles and random numbers do not depend on any velocity: the
// particles come from keyed permutations of the id ranks, and each pair
// draws from a stream of its own (twelve uniforms for Z, then the azimuth).
// So a cell's warp first derives them for 32 pairs at a time, flattened over
// all the cell's classes, and then applies the pairs in waves that the
// sequential definition allows to run side by side: the regular pairs of a
// species with itself (disjoint), each pair of an odd count's closing triple
// alone, and each round of N_fewer pairs of two species (disjoint) in turn.
// ---------------------------------------------------------------------

// Pseudo-random permutation of [0, n): four Feistel rounds (Luby and Rackoff)
// on 2h bits, 4^h >= n, with an integer mixing round function, walked back
// into [0, n) by cycle walking (Black and Rogaway, 2002).  The walk ends
// within 4^h steps because x itself lies in [0, n).
__device__ __forceinline__ uint32_t fe_round(uint32_t x, uint32_t k) {
    uint32_t t = (x ^ k) * 0x9E3779B1u;
    t ^= t >> 15;
    t *= 0x85EBCA77u;
    t ^= t >> 13;
    return t;
}
// h of the permutation of [0, n): the least h >= 1 with 4^h >= n
__device__ __forceinline__ int perm_bits(uint32_t n) {
    int h = 1;
    while ((1ull << (2 * h)) < (unsigned long long)n) ++h;
    return h;
}
// one pass of the four Feistel rounds on 2h bits
__device__ __forceinline__ uint32_t feistel4(uint32_t y, const uint4& key, int h) {
    const uint32_t mask = (1u << h) - 1u;
    uint32_t L = y >> h, R = y & mask;
    const uint32_t k4[4] = {key.x, key.y, key.z, key.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint32_t F = fe_round(R, k4[r]) & mask;
        const uint32_t t = L ^ F;
        L = R;
        R = t;
    }
    return (L << h) | R;
}
// Indices x0 and x1 under two permutations (or the same one twice), each
// walked back into its range [0, n) by repeating the rounds until the value
// falls in it; the two walks advance side by side.  A walk ends within 4^h
// steps, x lying in [0, n) itself (x is returned after 4^h, which it never
// reaches).
__device__ void perm_index2(uint32_t x0, uint32_t n0, const uint4& key0, int h0, uint32_t x1, uint32_t n1,
                            const uint4& key1, int h1, uint32_t& out0, uint32_t& out1) {
    const unsigned long long lim0 = 1ull << (2 * h0), lim1 = 1ull << (2 * h1);
    const unsigned long long lim = lim0 > lim1 ? lim0 : lim1;
    uint32_t y0 = x0, y1 = x1;
    bool d0 = false, d1 = false;
    out0 = x0;
    out1 = x1;
    for (unsigned long long it = 0; it < lim && !(d0 && d1); ++it) {
        if (!d0) {
            y0 = feistel4(y0, key0, h0);
            if (y0 < n0) {
                out0 = y0;
                d0 = true;
            } else if (it + 1 >= lim0) {
                d0 = true;
            }
        }
        if (!d1) {
            y1 = feistel4(y1, key1, h1);
            if (y1 < n1) {
                out1 = y1;
                d1 = true;
            } else if (it + 1 >= lim1) {
                d1 = true;
            }
        }
    }
}

// uniform on [0, 1) from the top 24 bits of a draw (as Stream::u01)
__device__ __forceinline__ float u01_of(uint32_t x) { return __fmul_rn((float)(x >> 8), 5.9604644775390625e-08f); }

// The draws of one Coulomb pair from its stream: Z (the Irwin-Hall sum of
// the first twelve uniforms, three Philox blocks) and the azimuth (points of
// the square from the following blocks, two per block, until one falls in
// the unit disc; fail after 64 tries, as azimuth()).  The three blocks of Z
// and the first block of the azimuth (which serves all but about one pair in
// twenty) are independent chains of rounds, computed side by side.
__device__ void coul_draws(uint32_t subject, uint32_t step, uint32_t sid, uint32_t seed, uint32_t run, float& z,
                           float& c, float& s, bool& fail) {
    const uint2 key = make_uint2(seed, run);
    const uint4 r0 = philox4x32_10(make_uint4(subject, step, sid, 0u), key);
    const uint4 r1 = philox4x32_10(make_uint4(subject, step, sid, 1u), key);
    const uint4 r2 = philox4x32_10(make_uint4(subject, step, sid, 2u), key);
    uint4 r = philox4x32_10(make_uint4(subject, step, sid, 3u), key);
    float zz = 0.0f;
    zz = zz + u01_of(r0.x);
    zz = zz + u01_of(r0.y);
    zz = zz + u01_of(r0.z);
    zz = zz + u01_of(r0.w);
    zz = zz + u01_of(r1.x);
    zz = zz + u01_of(r1.y);
    zz = zz + u01_of(r1.z);
    zz = zz + u01_of(r1.w);
    zz = zz + u01_of(r2.x);
    zz = zz + u01_of(r2.y);
    zz = zz + u01_of(r2.z);
    zz = zz + u01_of(r2.w);
    z = zz - 6.0f;
    fail = false;
#pragma unroll 1
    for (uint32_t b = 0; b < 32u; ++b) {
        if (b > 0u) r = philox4x32_10(make_uint4(subject, step, sid, 3u + b), key);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float u1 = 2.0f * u01_of(h ? r.z : r.x) - 1.0f;
            const float u2 = 2.0f * u01_of(h ? r.w : r.y) - 1.0f;
            const float q = u1 * u1 + u2 * u2;
            if (q < 1.0f && q > 0.0f) {
                const float rq = sqrtf(q);
                c = u1 / rq;
                s = u2 / rq;
                return;
            }
        }
    }
    fail = true;
    c = 1.0f;
    s = 0.0f;
}

// One pair's turn (after its draws): false when u = 0 (nothing to turn).
__device__ __forceinline__ bool coulomb_turn(V3& va, V3& vb, float Kn, float fa, float fb_, float z, float cph,
                                             float sph) {
    const float ux = va.x - vb.x, uy = va.y - vb.y, uz = va.z - vb.z;
    const float u2 = (ux * ux + uy * uy) + uz * uz;
    if (!(u2 > 0.0f)) return false;
    const float u = sqrtf(u2);
    float var = Kn / (u2 * u);
    var = var < 1e30f ? var : 1e30f;                // u -> 0: keep delta finite
    const float d = sqrtf(var) * z;
    // sin(theta) = 2 delta / (1 + delta^2), 1 - cos(theta) = 2 delta^2 / (1 + delta^2)
    float sth, omc;
    const float ad = d < 0.0f ? -d : d;
    if (ad <= 1.0f) {
        const float d2 = d * d, den = 1.0f + d2;
        sth = (2.0f * d) / den;
        omc = (2.0f * d2) / den;
    } else {
        const float rr = 1.0f / d, r2 = rr * rr, den = 1.0f + r2;
        sth = (2.0f * rr) / den;
        omc = 2.0f / den;
    }
    const float sc = sth * cph, ss = sth * sph;
    const float up = sqrtf(ux * ux + uy * uy);
    float dx, dy, dz;
    if (up > 0.0f) {
        const float a1 = ux / up, a2 = uy / up;
        dx = ((a1 * uz) * sc - (a2 * u) * ss) - ux * omc;
        dy = ((a2 * uz) * sc + (a1 * u) * ss) - uy * omc;
        dz = -(up * sc) - uz * omc;
    } else {                                         // u along the third axis
        dx = uz * sc;
        dy = uz * ss;
        dz = -(uz * omc);
    }
    va.x = va.x + fa * dx; va.y = va.y + fa * dy; va.z = va.z + fa * dz;
    vb.x = vb.x - fb_ * dx; vb.y = vb.y - fb_ * dy; vb.z = vb.z - fb_ * dz;
    return true;
}

// Classes of a cell: 0 the electrons with themselves, 1 + i the electrons
// with ion species i (Cu+, Cu2+ SW, Cu2+ DI, Cu3+, Cu4+), on heavy steps
// 6.. the ion species a <= b (in order).  Lists: 0 the electrons, 1 + i ion
// species i.
constexpr int COUL_NCLS = 21;
constexpr int COUL_NLIST = 6;
// charged particles of a cell whose velocities its warp holds in shared
// memory (in the words of its rank-table sort buffer, free once the tables
// are built)
constexpr int COUL_CACHE = 384;
constexpr int COUL_WARPS = 4;           // warps of a k_coulomb block
// words of a warp's buffer: the rank-table sort of a register-cached list,
// then the velocity cache (three floats and a flag byte per particle)
constexpr int COUL_SORT_WORDS = 4 * RANK_WARP_MAX + 256, COUL_CACHE_WORDS = (COUL_CACHE * 13 + 3) / 4;
constexpr int COUL_SBUF = COUL_SORT_WORDS > COUL_CACHE_WORDS ? COUL_SORT_WORDS : COUL_CACHE_WORDS;

struct CoulClass {
    uint4 k1, k2;          // permutation keys: of the one species; or of the more and the fewer
    float Kn, fa, fb;
    uint32_t start;        // first pair in the cell's flattened order
    uint32_t npairs;
    uint32_t P;            // one species: regular pairs; two: the fewer's count (a round)
    uint32_t N;            // one species: its count; two: the more numerous's
    uint8_t la, lb;        // the lists of the pair's first and second particle
    uint8_t cls, a_many;   // a_many: list la is the more numerous (la on a tie)
};
struct CoulWarp {
    CoulClass cl[COUL_NCLS];
    uint32_t base[COUL_NLIST], n[COUL_NLIST];
    uint32_t coff[COUL_NLIST], cn[COUL_NLIST];   // a list's place and count in the velocity cache
    uint32_t sorted;       // bit l: list l's ids ascend (rank = position)
};

__device__ __forceinline__ void class_lists(int t, int& la, int& lb) {
    if (t == 0) {
        la = lb = 0;
    } else if (t < 6) {
        la = 0;
        lb = t;
    } else {
        int idx = t - 6, a = 0;
        while (idx >= 5 - a) {
            idx -= 5 - a;
            ++a;
        }
        la = 1 + a;
        lb = 1 + a + idx;
    }
}
__device__ __forceinline__ int list_species(int l) { return l == 0 ? SP_E : SP_CUP + l - 1; }

// The Coulomb pairs (after all cells' DSMC classes: cells are independent,
// so this is the order of cell-by-cell processing): one warp per cell with
// charged particles, grid-stride over the cells, on the lists of the step's
// start; a particle whose species changed this step is left out.
__global__ void __launch_bounds__(128, 6) k_coulomb(Particles A, RankScratch S, const uint32_t* __restrict__ off,
                                                   const uint32_t* __restrict__ cnt, DevState* st, KParams P,
                                                   CollConsts cc, const double* __restrict__ cw) {
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    __shared__ uint32_t s_sort[COUL_WARPS][COUL_SBUF];   // per-warp rank-table sort, then velocity cache
    __shared__ CoulWarp s_cw[COUL_WARPS];
    const int lane = threadIdx.x & 31;
    const int wib = (threadIdx.x >> 5) & (COUL_WARPS - 1);
    uint32_t* sbuf = s_sort[wib];
    CoulWarp& W = s_cw[wib];
    const uint32_t C = P.ncell;
    const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    for (uint32_t c = warp0; c < C; c += nwarps) {
        // the cell's charged lists (lane l reads list l)
        uint32_t nl = 0, bl = 0;
        if (lane < COUL_NLIST) {
            const int sp = list_species(lane);
            if (sp < P.nsp) {
                const uint32_t b = (uint32_t)sp * C + c;
                nl = cnt[b];
                bl = off[b];
            }
        }
        const uint32_t Ne = __shfl_sync(FULL, nl, 0);
        if (Ne == 0u && !P.heavy_step) continue;
        // the class table: lane t takes class t
        int la = 0, lb = 0;
        if (lane < COUL_NCLS) class_lists(lane, la, lb);
        const uint32_t Na = __shfl_sync(FULL, nl, la), Nb = __shfl_sync(FULL, nl, lb);
        bool on = false;
        uint32_t np = 0, Pk = 0, Nk = 0;
        bool a_many = true;
        if (lane < COUL_NCLS) {
            if (la == lb) {
                on = Na >= 2u && (lane == 0 || P.heavy_step);
                Pk = Na / 2u - (Na % 2u);
                np = Pk + (Na % 2u ? 3u : 0u);
                Nk = Na;
            } else {
                on = Na >= 1u && Nb >= 1u && (lane < 6 || P.heavy_step);
                a_many = Na >= Nb;
                Nk = a_many ? Na : Nb;
                Pk = a_many ? Nb : Na;
                np = Nk;
            }
        }
        const unsigned mact = __ballot_sync(FULL, on);
        if (mact == 0u) continue;
        const int r = run_of(P, c);
        const RunInfo* RI = &P.runs[r];
        const uint32_t lc = c - RI->cell_base;
        if (!on) np = 0;
        uint32_t incl = np;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += y;
        }
        const uint32_t T = __shfl_sync(FULL, incl, 31);
        const int nact = __popc(mact);
        if (on) {
            const uint32_t row = RI->row_base + lc % (uint32_t)RI->nr;
            const double w = lane < 6 ? cw[row] : cw[P.cw_heavy + row];
            const uint32_t Nf = la == lb ? Na : min(Na, Nb);
            CoulClass K;
            Stream ps(lc, st->step, SID_COUL_PERM | (uint32_t)lane, RI->seed, RI->run);
            K.k1 = make_uint4(ps.next(), ps.next(), ps.next(), ps.next());
            K.k2 = make_uint4(0u, 0u, 0u, 0u);
            if (la != lb) K.k2 = make_uint4(ps.next(), ps.next(), ps.next(), ps.next());
            K.Kn = (float)(cc.kc[lane] * (double)Nf * w);
            K.fa = lane >= 1 && lane < 6 ? cc.a_e : 0.5f;
            K.fb = lane >= 1 && lane < 6 ? cc.a_t : 0.5f;
            K.start = incl - np;
            K.npairs = np;
            K.P = Pk;
            K.N = Nk;
            K.la = (uint8_t)la;
            K.lb = (uint8_t)lb;
            K.cls = (uint8_t)lane;
            K.a_many = a_many ? 1 : 0;
            W.cl[__popc(mact & lt)] = K;
        }
        // lists any class uses: rank tables, then the velocities in shared
        // memory when they fit
        unsigned used = on ? ((1u << la) | (1u << lb)) : 0u;
        used = __reduce_or_sync(FULL, used);
        const uint32_t idn = P.rs[r].id_next;
        const int id_top = idn > 1u ? 31 - __clz((int)(idn - 1u)) : 0;
        uint32_t sorted = 0, tot = 0;
        for (int l = 0; l < COUL_NLIST; ++l) {
            const uint32_t n = __shfl_sync(FULL, nl, l), b = __shfl_sync(FULL, bl, l);
            const bool u = (used >> l) & 1u;
            if (lane == 0) {
                W.base[l] = b;
                W.n[l] = n;
                W.coff[l] = tot;
                W.cn[l] = u ? n : 0u;
            }
            if (!u) continue;
            tot += n;
            IdList L;
            load_ids(L, A.id, b, n, n, S, sbuf, lane, id_top, true);
            if (L.sorted) sorted |= 1u << l;
        }
        if (lane == 0) W.sorted = sorted;
        const bool cached = tot <= (uint32_t)COUL_CACHE;
        float* const cvz = reinterpret_cast<float*>(sbuf);
        float* const cvr = cvz + COUL_CACHE;
        float* const cvt = cvr + COUL_CACHE;
        uint8_t* const touched = reinterpret_cast<uint8_t*>(cvt + COUL_CACHE);
        __syncwarp();
        if (cached) {
            for (int l = 0; l < COUL_NLIST; ++l) {
                const uint32_t n = W.cn[l], b = W.base[l], co = W.coff[l];
                for (uint32_t q = (uint32_t)lane; q < n; q += 32) {
                    cvz[co + q] = A.vz[b + q];
                    cvr[co + q] = A.vr[b + q];
                    cvt[co + q] = A.vt[b + q];
                    touched[co + q] = 0;
                }
            }
        }
        __syncwarp();
        float* VZ = cached ? cvz : A.vz;
        float* VR = cached ? cvr : A.vr;
        float* VT = cached ? cvt : A.vt;
        uint32_t n_ee = 0, n_ei = 0, n_ii = 0, n_fb = 0;
        int jw = 0;                      // the class of the wave being applied
        for (uint32_t c0 = 0; c0 < T; c0 += 32) {
            // lane q: pair c0 + q's particles and draws
            const uint32_t p = c0 + (uint32_t)lane;
            uint32_t ia = 0, ib = 0;
            float z = 0.0f, cph = 1.0f, sph = 0.0f, Kn = 0.0f;
            bool valid = false, fail = false;
            if (p < T) {
                int j = 0;
                while (j + 1 < nact && W.cl[j + 1].start <= p) ++j;
                const CoulClass& K = W.cl[j];
                const uint32_t k = p - K.start;
                uint32_t ra, rb;
                Kn = K.Kn;
                if (K.la == K.lb) {
                    const uint32_t N = K.N;
                    const int h = perm_bits(N);
                    uint32_t xa = 2u * k, xb = 2u * k + 1u;
                    if (k >= K.P) {              // the closing triple: pair q joins q and q + 1 (mod 3)
                        const uint32_t q = k - K.P;
                        xa = N - 3u + q;
                        xb = N - 3u + (q + 1u) % 3u;
                        Kn = Kn * 0.5f;
                    }
                    perm_index2(xa, N, K.k1, h, xb, N, K.k1, h, ra, rb);
                } else {
                    uint32_t m, f;
                    perm_index2(k, K.N, K.k1, perm_bits(K.N), k % K.P, K.P, K.k2, perm_bits(K.P), m, f);
                    ra = K.a_many ? m : f;
                    rb = K.a_many ? f : m;
                }
                const int la_ = K.la, lb_ = K.lb;
                const uint32_t na = W.n[la_], nb = W.n[lb_], ba = W.base[la_], bb = W.base[lb_];
                const uint32_t pa = (W.sorted >> la_) & 1u ? ra : S.table[ba + ra];
                const uint32_t pb = (W.sorted >> lb_) & 1u ? rb : S.table[bb + rb];
                // the draws do not depend on the particles: they are computed
                // while the rank lookups are in flight (and dropped for a pair
                // that does not take place)
                coul_draws(lc, st->step, sid_coul(K.cls, k), RI->seed, RI->run, z, cph, sph, fail);
                if (pa < na && pb < nb) {
                    const uint32_t ka = A.key[ba + pa], kb = A.key[bb + pb];
                    valid = !(ka & KEY_FLAG) && (int)key_species(ka) == list_species(la_) && !(kb & KEY_FLAG) &&
                            (int)key_species(kb) == list_species(lb_);
                    ia = cached ? W.coff[la_] + pa : ba + pa;
                    ib = cached ? W.coff[lb_] + pb : bb + pb;
                } else {
                    set_error(st, ERR_BOUNDS);   // ids not unique: corrupt state, never index with it
                }
                if (!valid) fail = false;
            }
            // the chunk's pairs in waves, in order
            const uint32_t c1 = min(c0 + 32u, T);
            for (uint32_t pw = c0; pw < c1;) {
                while (pw >= W.cl[jw].start + W.cl[jw].npairs) ++jw;
                const CoulClass& K = W.cl[jw];
                const uint32_t k = pw - K.start;
                uint32_t we;
                if (K.la == K.lb) we = k < K.P ? K.start + K.P : pw + 1u;
                else we = K.start + min((k / K.P + 1u) * K.P, K.N);
                const uint32_t e = min(we, c1);
                const int src = (int)(pw - c0) + lane;
                const uint32_t wa = __shfl_sync(FULL, ia, src & 31), wb = __shfl_sync(FULL, ib, src & 31);
                const float wz = __shfl_sync(FULL, z, src & 31), wc = __shfl_sync(FULL, cph, src & 31);
                const float ws = __shfl_sync(FULL, sph, src & 31), wk = __shfl_sync(FULL, Kn, src & 31);
                const bool wv = __shfl_sync(FULL, valid, src & 31), wf = __shfl_sync(FULL, fail, src & 31);
                if (pw + (uint32_t)lane < e && wv) {
                    V3 va{VZ[wa], VR[wa], VT[wa]}, vb{VZ[wb], VR[wb], VT[wb]};
                    if (coulomb_turn(va, vb, wk, K.fa, K.fb, wz, wc, ws)) {
                        VZ[wa] = va.x; VR[wa] = va.y; VT[wa] = va.z;
                        VZ[wb] = vb.x; VR[wb] = vb.y; VT[wb] = vb.z;
                        if (cached) {
                            touched[wa] = 1;
                            touched[wb] = 1;
                        }
                        if (K.cls == 0) ++n_ee;
                        else if (K.cls < 6) ++n_ei;
                        else ++n_ii;
                        if (wf) ++n_fb;
                    }
                }
                __syncwarp();
                pw = e;
            }
        }
        if (cached) {
            // the velocities the pairs changed back to their slots
            for (uint32_t i = (uint32_t)lane; i < tot; i += 32) {
                if (!touched[i]) continue;
                int l = 0;
                while (i >= W.coff[l] + W.cn[l]) ++l;
                const uint32_t slot = W.base[l] + (i - W.coff[l]);
                A.vz[slot] = cvz[i];
                A.vr[slot] = cvr[i];
                A.vt[slot] = cvt[i];
            }
        }
        __syncwarp();
        const uint32_t ee = __reduce_add_sync(FULL, n_ee), ei = __reduce_add_sync(FULL, n_ei);
        const uint32_t ii = __reduce_add_sync(FULL, n_ii), fb = __reduce_add_sync(FULL, n_fb);
        if (lane == 0) {
            RunState& rsv = P.rs[r];
            if (ee) atomicAdd(&rsv.ctr[C_COUL_EE], (unsigned long long)ee);
            if (ei) atomicAdd(&rsv.ctr[C_COUL_EI], (unsigned long long)ei);
            if (ii) atomicAdd(&rsv.ctr[C_COUL_II], (unsigned long long)ii);
            if (fb) atomicAdd(&rsv.ctr[C_ISOFB], (unsigned long long)fb);
        }
    }
}

template <bool EXT>
__global__ void __launch_bounds__(128, 3) k_collide(Particles A, RankScratch S, const uint32_t* __restrict__ off,
                                                 const uint32_t* __restrict__ cnt,
                                                 const uint4* __restrict__ nc, const uint4* __restrict__ nc2,
                                                 const uint32_t* __restrict__ cand_off,
                                                 const uint32_t* __restrict__ active, DevState* st, long long* rho_e,
                                                 long long* rho_h, const float* __restrict__ xsE,
                                                 const float* __restrict__ xs, const double* __restrict__ cw,
                                                 KParams P, CollConsts cc, uint32_t nbins) {
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    __shared__ uint32_t s_sort[4][4 * RANK_WARP_MAX + 256];   // per-warp rank-table sort
    const int lane = threadIdx.x & 31;
    uint32_t* sbuf = s_sort[(threadIdx.x >> 5) & 3];
    const uint32_t C = P.ncell;
    const uint32_t n_heavy = st->n_heavy, n_light = st->n_light;
    const uint32_t n_alive = (uint32_t)st->tail_base;   // spawn slots follow the bins
    // heavy cells first, taken one at a time from a shared cursor by the
    // first min(n_heavy, warps) warps; then the light cells, warp-strided
    const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    bool heavy_phase = warp0 < n_heavy;
    uint32_t wl = warp0;
    for (;;) {
        uint32_t c = 0;
        if (heavy_phase) {
            uint32_t w = 0;
            if (lane == 0) w = atomicAdd(&st->collide_next, 1u);
            w = __shfl_sync(FULL, w, 0);
            if (w < n_heavy) c = active[w];
            else heavy_phase = false;
        }
        if (!heavy_phase) {
            if (wl >= n_light) break;
            c = active[C - 1u - wl];
            wl += nwarps;
        }
        const uint4 n = nc[c];         // candidates of the classes (e,Cu), (e,Cu+), (Cu,Cu+), (Cu,Cu)
        // and of (e,Cu2+ SW), (e,Cu2+ DI), (e,Cu3+)
        const uint4 n2 = EXT && P.charge_max >= 3 ? nc2[c] : make_uint4(0u, 0u, 0u, 0u);
        const int r = run_of(P, c);
        const RunInfo* RI = &P.runs[r];
        const uint32_t lc = c - RI->cell_base;
        CellCtx cx;
        cx.cell = c;
        cx.RI = RI;
        cx.geom = P.geom;
        cx.nres = 2u * (n.x + n.y + n2.x + n2.y + n2.z);
        cx.slot0 = (unsigned long long)n_alive + 2ull * cand_off[c];
        // ids: the run's next id plus twice the candidates of the run's earlier cells
        cx.id0 = P.rs[r].id_next + 2u * (cand_off[c] - cand_off[RI->cell_base]);
        // every id in the cell's lists is below the run's next id
        const uint32_t idn = P.rs[r].id_next;
        const int id_top = idn > 1u ? 31 - __clz((int)(idn - 1u)) : 0;
        cx.s = 0;
        for (int q = 0; q < NCH; ++q) cx.ev[q] = 0;
        cx.nulls = cx.consumed = cx.thr = cx.viol = cx.fb = 0;
        cx.coul_ee = cx.coul_ei = cx.coul_ii = 0;
        if (cx.slot0 + cx.nres > P.capacity) {
            // no room for this cell's spawns: report, and leave its reserved
            // slots (those that exist) dead
            if (lane == 0) set_error(st, ERR_CAPACITY);
            for (unsigned long long q = cx.slot0 + lane; q < P.capacity && q < cx.slot0 + cx.nres; q += 32)
                A.key[q] = DEAD;
            continue;
        }
        const uint32_t e_base = off[c];
        const uint32_t Ne = cnt[c];
        // lookups of each list over all classes (the rank-table decisions of
        // k_ncand use the same totals): the Coulomb pairs look up every
        // electron and every ion of a cell with electrons
        // (ion pairs collide on heavy steps even where there are no electrons)
        const bool coul_e = EXT && P.coulomb && Ne > 0;
        const bool coul = EXT && P.coulomb && (Ne > 0 || P.heavy_step);
        const uint32_t look_e = n.x + n.y + n2.x + n2.y + n2.z + (coul_e ? Ne : 0u);
        const uint32_t look_cu = n.x + n.z + 2u * n.w, look_ci = n.y + n.z;
        // the first list of a pair: electrons for the electron classes, Cu for
        // the heavy classes (loaded over the electrons' list once those are done)
        IdList el;
        uint32_t a_base = e_base, Na = Ne;
        bool cu_first = false;
        if (look_e) load_ids(el, A.id, e_base, Ne, look_e, S, sbuf, lane, id_top);
        for (int k = 0; k < (EXT ? NCLS : 2); ++k) {
            const uint32_t ncand = k == 0 ? n.x : k == 1 ? n.y : k == 2 ? n2.x : k == 3 ? n2.y : k == 4 ? n2.z
                                 : k == 5 ? n.z : n.w;
            if (ncand == 0) continue;
            if (k >= NECLS && !cu_first) {
                cu_first = true;
                a_base = off[C + c];
                Na = cnt[C + c];
                load_ids(el, A.id, a_base, Na, look_cu, S, sbuf, lane, id_top);
            }
            const int ts = class_target(k);
            const uint32_t tb = (uint32_t)ts * C + c;
            const uint32_t t_base = off[tb];
            const uint32_t Nt = cnt[tb];
            // the target list's lookups over every class that draws from it
            const uint32_t t_look = ts == SP_CU ? look_cu : (ts == SP_CUP ? look_ci : ncand) + (coul ? Nt : 0u);
            IdList tl;
            load_ids(tl, A.id, t_base, Nt, t_look, S, sbuf, lane, id_top);
            // candidates in batches of 32: lane q draws candidate m0 + q's pair and
            // prefetches its particles; lane 0 then applies them in order,
            // re-reading a candidate whose particles an earlier candidate of
            // the batch may have changed
            for (uint32_t m0 = 0; m0 < ncand; m0 += 32) {
                const uint32_t nb = min(32u, ncand - m0);
                const bool has = (uint32_t)lane < nb;
                uint32_t i = 0, j = 0;
                float Racc = 0.0f, Rch = 0.0f;
                if (has) {
                    Stream rs(lc, st->step, sid_cand(k, m0 + lane), RI->seed, RI->run);
                    i = rs.pick(Na);
                    if (k == 6) {           // a second, different Cu
                        j = rs.pick(Na - 1u);
                        if (j >= i) ++j;
                    } else {
                        j = rs.pick(Nt);
                    }
                    Racc = rs.u01();
                    Rch = rs.u01();
                }
                uint32_t pe = 0, pt = 0;
                if (el.sorted) {
                    pe = i;
                } else if (el.table) {
                    if (has) pe = el.table[i];
                } else {
                    for (uint32_t q = 0; q < nb; ++q) {
                        const uint32_t p = select_rank_list(el, __shfl_sync(FULL, i, (int)q), lane);
                        if ((uint32_t)lane == q) pe = p;
                    }
                }
                if (tl.sorted) {
                    pt = j;
                } else if (tl.table) {
                    if (has) pt = tl.table[j];
                } else {
                    for (uint32_t q = 0; q < nb; ++q) {
                        const uint32_t p = select_rank_list(tl, __shfl_sync(FULL, j, (int)q), lane);
                        if ((uint32_t)lane == q) pt = p;
                    }
                }
                const bool ok = has && pe < Na && pt < Nt;   // ids not unique: corrupt state, never index with it
                if (has && !ok) set_error(st, ERR_BOUNDS);
                const uint32_t ie = a_base + (ok ? pe : 0u), it = t_base + (ok ? pt : 0u);
                uint32_t tkey = 0, akey = 0;
                V3 ve{0.0f, 0.0f, 0.0f}, vt{0.0f, 0.0f, 0.0f};
                if (ok) {
                    tkey = A.key[it];
                    if (k >= NECLS) akey = A.key[ie];
                    ve = V3{A.vz[ie], A.vr[ie], A.vt[ie]};
                    vt = V3{A.vz[it], A.vr[it], A.vt[it]};
                }
                // cross sections of every lane's pair, in parallel (redone by
                // lane 0 for a pair an earlier candidate may have changed)
                const PairEval ev = evaluate_pair(k, ve, vt, xsE, xs, cc);
                // dirty: shares a particle with an earlier candidate of the batch
                // (the two particles of a (Cu, Cu) pair come from one list)
                bool dirty = false;
                for (uint32_t q = 0; q + 1 < nb; ++q) {
                    const uint32_t e2 = __shfl_sync(FULL, ie, (int)q), t2 = __shfl_sync(FULL, it, (int)q);
                    if (q < (uint32_t)lane && (e2 == ie || t2 == it || (k == 6 && (e2 == it || t2 == ie))))
                        dirty = true;
                }
                // a candidate no earlier one of the batch touches sees the
                // particles as prefetched: its lane takes the target and
                // acceptance tests (the same float operations lane 0 would),
                // and only accepted or touched candidates go through lane 0,
                // in candidate order
                const bool cons = consumed_pair(k, akey, tkey);
                const bool acc = !cons && Racc * cc.sgmax[k] < ev.sg;
                const bool clean = ok && !dirty;
                const unsigned m_cons = __ballot_sync(FULL, clean && cons);
                const unsigned m_viol = __ballot_sync(FULL, clean && !cons && ev.sg > cc.sgmax[k]);
                const unsigned m_null = __ballot_sync(FULL, clean && !cons && !acc);
                if (lane == 0) {
                    cx.consumed += (uint32_t)__popc(m_cons);
                    cx.viol += (uint32_t)__popc(m_viol);
                    cx.nulls += (uint32_t)__popc(m_null);
                }
                const unsigned todo = __ballot_sync(FULL, ok && (dirty || acc));
                for (unsigned mq = todo; mq; mq &= mq - 1u) {
                    const uint32_t q = (uint32_t)(__ffs(mq) - 1);
                    const bool dq = __shfl_sync(FULL, dirty, (int)q);
                    const uint32_t ieq = __shfl_sync(FULL, ie, (int)q), itq = __shfl_sync(FULL, it, (int)q);
                    uint32_t tkq = __shfl_sync(FULL, tkey, (int)q), akq = __shfl_sync(FULL, akey, (int)q);
                    V3 veq{__shfl_sync(FULL, ve.x, (int)q), __shfl_sync(FULL, ve.y, (int)q),
                           __shfl_sync(FULL, ve.z, (int)q)};
                    V3 vtq{__shfl_sync(FULL, vt.x, (int)q), __shfl_sync(FULL, vt.y, (int)q),
                           __shfl_sync(FULL, vt.z, (int)q)};
                    const float Ra = __shfl_sync(FULL, Racc, (int)q), Rc = __shfl_sync(FULL, Rch, (int)q);
                    PairEval evq;
#pragma unroll
                    for (int e = 0; e < 4; ++e) evq.cum[e] = __shfl_sync(FULL, ev.cum[e], (int)q);
                    evq.sg = __shfl_sync(FULL, ev.sg, (int)q);
                    if (lane == 0) {
                        if (dq) {
                            tkq = A.key[itq];
                            if (k >= NECLS) akq = A.key[ieq];
                            veq = V3{A.vz[ieq], A.vr[ieq], A.vt[ieq]};
                            vtq = V3{A.vz[itq], A.vr[itq], A.vt[itq]};
                            evq = evaluate_pair(k, veq, vtq, xsE, xs, cc);
                        }
                        // the candidate's stream after its four pair-choice draws
                        Stream rs(lc, st->step, sid_cand(k, m0 + q), RI->seed, RI->run);
                        rs.ctr.w = 1u;
                        rs.used = 4;
                        if (k < NECLS)
                            process_candidate(A, cx, rs, k, ieq, itq, tkq, veq, vtq, evq, Ra, Rc, xsE, xs, cc, st,
                                              rho_e, rho_h, !dq);
                        else
                            process_heavy_pair(A, cx, rs, k, ieq, itq, akq, tkq, veq, vtq, evq, Ra, cc, !dq);
                    }
                }
                __syncwarp();
            }
        }
        const uint32_t s = __shfl_sync(FULL, cx.s, 0);
        for (uint32_t q = s + lane; q < cx.nres; q += 32) A.key[cx.slot0 + q] = DEAD;
        if (lane == 0) {
            RunState& rsv = P.rs[r];
            for (int q = 0; q < NCH; ++q)
                if (cx.ev[q]) atomicAdd(&rsv.ctr[c_event(q)], (unsigned long long)cx.ev[q]);
            if (cx.nulls) atomicAdd(&rsv.ctr[C_NULL], (unsigned long long)cx.nulls);
            if (cx.consumed) atomicAdd(&rsv.ctr[C_CONSUMED], (unsigned long long)cx.consumed);
            if (cx.thr) atomicAdd(&rsv.ctr[C_THR], (unsigned long long)cx.thr);
            if (cx.viol) atomicAdd(&rsv.ctr[C_VIOL], (unsigned long long)cx.viol);
            if (cx.fb) atomicAdd(&rsv.ctr[C_ISOFB], (unsigned long long)cx.fb);
        }
    }
}

// slot / id bookkeeping of the step and the RC circuit of each run
__global__ void k_finalize(const uint32_t* __restrict__ off, uint32_t nbins, const uint32_t* __restrict__ cand_off,
                           DevState* st, KParams P, const RunCircuit* __restrict__ circ, double dt, int circuit) {
    const uint32_t C = P.ncell;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long T = cand_off[C];
        unsigned long long ns = st->tail_base + 2ull * T;
        if (ns > P.capacity) {
            set_error(st, ERR_CAPACITY);
            ns = P.capacity;
        }
        // the next step's particles (in bins and in the spawn slots) within
        // the configured capacity
        if (st->n_live + st->n_e + 2ull * T > P.user_capacity) set_error(st, ERR_CAPACITY);
        st->n_slots = ns;
        st->n_bigc = 0;
        st->n_ovf = 0;
        st->since += 1u;
        st->n_heavy = 0;
        st->n_light = 0;
        st->n_mid = 0;
        st->n_big = 0;
        st->collide_next = 0;
        st->n_sput = 0;
    }
    // the step is over for every kernel that draws from it
    if (blockIdx.x == 0 && threadIdx.x == 0) st->step += 1u;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P.nruns; r += gridDim.x * blockDim.x) {
        const RunInfo& RI = P.runs[r];
        RunState& rs = P.rs[r];
        const unsigned long long T = cand_off[RI.cell_base + RI.ncell] - cand_off[RI.cell_base];
        if ((unsigned long long)rs.id_next + 2ull * T > 0xFFFFFFFFull) set_error(st, ERR_IDS);
        rs.id_next += (uint32_t)(2ull * T);
        rs.ctr[C_CAND] += T;
        if (circuit) {
            // C dV/dt = (V0 - V)/R - I_gap; the gap current leaves the anode node
            const double I = -rs.anode_charge_step / dt;
            rs.I_gap = I;
            rs.V += dt / circ[r].C_farad * ((circ[r].V0 - rs.V) / circ[r].R_ohm - I);
            rs.anode_charge_step = 0.0;
        }
    }
}

// ---------------------------------------------------------------------
// cathode injection (Sec. 2.3): FN electrons from the tip and neutrals at
// a fixed fraction of the electron flux; one block per run.
// ---------------------------------------------------------------------
__device__ __forceinline__ float rayleigh(const float* __restrict__ ray, float U) {
    const float x = U * 1023.0f;
    const int k = min((int)x, 1022);
    const float t = x - (float)k;
    return ray[k] + t * (ray[k + 1] - ray[k]);
}

__global__ void __launch_bounds__(256) k_inject(Particles A, const float2* __restrict__ E, DevState* st, KParams P,
                                                const InjectConsts* __restrict__ icv, const float* __restrict__ ray) {
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    __shared__ uint32_t ne_s[64], nn_s[64], pre_s[65];
    __shared__ unsigned long long slot0_s;
    const int run = blockIdx.x;
    const InjectConsts& ic = icv[run];
    const RunInfo& RI = P.runs[run];
    RunState& rs = P.rs[run];
    if (ic.ntip == 0) return;
    const int t = threadIdx.x;
    if (t < ic.ntip) {
        const int j = t;
        const double ezs = 0.5 * ((double)E[node_of(RI, 0, 0, j)].x + (double)E[node_of(RI, 0, 0, j + 1)].x);
        const double F = ic.beta * (ezs < 0 ? -ezs : 0.0);
        double J = 0.0;
        if (F > 0.0) {
            const double Afn = 1.541434e-6, Bfn = 6.830890e9;
            J = Afn / ic.work * F * F * exp(-Bfn * ic.work * sqrt(ic.work) / F);
        }
        const double lam_e = J * ic.area[j] * ic.dt / (1.602176634e-19 * ic.weight);
        const double lam_n = ic.ratio * lam_e;
        Stream s((uint32_t)j, st->step, SID_INJ_COUNT, RI.seed, RI.run);
        const double Re = (double)s.u01(), Rn = (double)s.u01();
        ne_s[j] = (uint32_t)floor(lam_e + Re);
        nn_s[j] = (uint32_t)floor(lam_n + Rn);
    }
    __syncthreads();
    if (t == 0) {
        uint32_t acc = 0;
        for (int j = 0; j < ic.ntip; ++j) {
            pre_s[j] = acc;
            acc += ne_s[j] + nn_s[j];
        }
        pre_s[ic.ntip] = acc;
        slot0_s = acc ? atomicAdd(&st->n_slots, (unsigned long long)acc) : 0ull;
    }
    __syncthreads();
    const uint32_t total = pre_s[ic.ntip];
    const unsigned long long slot0 = slot0_s;
    const uint32_t id0 = rs.id_next;
    uint32_t emitted_e = 0, emitted_cu = 0;
    uint32_t fb = 0;
    for (uint32_t p = t; p < total; p += blockDim.x) {
        int j = 0;
        while (pre_s[j + 1] <= p) ++j;
        const uint32_t loc = p - pre_s[j];
        const bool is_e = loc < ne_s[j];
        Stream sp((uint32_t)j, st->step, is_e ? sid_inj_e(loc) : sid_inj_cu(loc - ne_s[j]), RI.seed, RI.run);
        const float U = sp.u01();
        const float lo = ic.lo[j], hi = ic.hi[j];
        const float rr = sqrtf(lo * lo + U * (hi * hi - lo * lo));
        float pr = rr - lo;
        if (pr >= 1.0f) pr = 0x1.fffffep-1f;
        if (pr < 0.0f) pr = 0.0f;
        float vz = 0.f, vr = 0.f, vt = 0.f;
        if (!is_e) {
            const float U1 = sp.u01(), U2 = sp.u01();
            vz = ic.vth * rayleigh(ray, U1);
            const float s = ic.vth * rayleigh(ray, U2);
            float cp, sn;
            azimuth(sp, cp, sn, fb);
            vr = s * cp;
            vt = s * sn;
        }
        const unsigned long long slot = slot0 + p;
        if (slot >= P.capacity) {
            set_error(st, ERR_CAPACITY);
            continue;
        }
        A.key[slot] = make_key(is_e ? SP_E : SP_CU, RI.cell_base + (uint32_t)j);   // iz = 0
        A.pz[slot] = 0.0f;
        A.pr[slot] = pr;
        A.vz[slot] = vz;
        A.vr[slot] = vr;
        A.vt[slot] = vt;
        A.id[slot] = id0 + p;
        if (is_e) ++emitted_e; else ++emitted_cu;
    }
    if (emitted_e) {
        atomicAdd(&rs.ctr[C_EMIT_E], (unsigned long long)emitted_e);
        for (uint32_t q = 0; q < emitted_e; ++q) atomicAdd(&rs.charge_cathode, 1.602176634e-19 * ic.weight);
    }
    if (emitted_cu) atomicAdd(&rs.ctr[C_EMIT_CU], (unsigned long long)emitted_cu);
    if (fb) atomicAdd(&rs.ctr[C_ISOFB], (unsigned long long)fb);
    __syncthreads();
    if (t == 0) {
        rs.id_next = id0 + total;
        if (slot0 + total > P.capacity) atomicMin(&st->n_slots, P.capacity);
    }
}

constexpr size_t RT_SMEM = (size_t)RANK_BLOCK_MAX * 4 * sizeof(uint32_t);
constexpr size_t RT_MID_SMEM = (size_t)RANK_MID_MAX * 4 * sizeof(uint32_t);

// ---------------------------------------------------------------------
// Ion-impact sputtering (Sec. 2.3), after the push: each run's block takes
// the impacts the push recorded for it, sorts them by the ion's id, and
// appends their atoms after the slots in use, as movers that the sort which
// follows places, with ids from the run's next id in that order.  An atom leaves the
// impact point on the electrode surface with an effusive flux at
// sputter_T: Rayleigh normal and transverse speeds, uniform azimuth.
// ---------------------------------------------------------------------
constexpr int SPUT_THREADS = 1024;
constexpr uint32_t SPUT_MAX = 8192;              // impacts per run and step
constexpr size_t SPUT_SMEM = SPUT_MAX * sizeof(unsigned long long);

__global__ void __launch_bounds__(SPUT_THREADS) k_sputter(Particles M, uint32_t* mm, DevState* st, KParams P,
                                                          const float* __restrict__ ray, uint32_t* in_cnt) {
    if (st->error) return;                           // a fault was flagged: the state is not stepped further
    extern __shared__ unsigned long long s_key[];    // ion id << 32 | record index
    __shared__ uint32_t s_cnt, s_el[2], s_wsum[SPUT_THREADS / 32];
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_id0, s_ok;
    const int r = blockIdx.x;
    const uint32_t tid = threadIdx.x;
    const uint32_t nq = min(st->n_sput, P.squeue_cap);
    if (tid == 0) {
        s_cnt = 0u;
        s_el[0] = s_el[1] = 0u;
    }
    __syncthreads();
    for (uint32_t x = tid; x < nq; x += SPUT_THREADS) {
        const SputRec rec = P.squeue[x];
        if ((int)(rec.meta >> 1) != r) continue;
        const uint32_t k = atomicAdd(&s_cnt, 1u);
        if (k < SPUT_MAX) s_key[k] = ((unsigned long long)rec.id << 32) | x;
    }
    __syncthreads();
    const uint32_t m = s_cnt;
    if (m == 0u) return;
    if (m > SPUT_MAX) {
        if (tid == 0) set_error(st, ERR_CAPACITY);
        return;
    }
    // bitonic sort of the keys, padded with all-ones to a power of two
    uint32_t np2 = 1u;
    while (np2 < m) np2 <<= 1;
    for (uint32_t x = m + tid; x < np2; x += SPUT_THREADS) s_key[x] = ~0ull;
    __syncthreads();
    for (uint32_t kk = 2u; kk <= np2; kk <<= 1)
        for (uint32_t j = kk >> 1; j > 0u; j >>= 1) {
            for (uint32_t x = tid; x < np2; x += SPUT_THREADS) {
                const uint32_t y = x ^ j;
                if (y > x) {
                    const unsigned long long a = s_key[x], b = s_key[y];
                    if ((a > b) == ((x & kk) == 0u)) {
                        s_key[x] = b;
                        s_key[y] = a;
                    }
                }
            }
            __syncthreads();
        }
    // atoms per impact in id order: each thread a contiguous chunk, an
    // exclusive scan of the chunk sums across the block
    const uint32_t per = (m + SPUT_THREADS - 1u) / SPUT_THREADS;
    const uint32_t c0 = min(tid * per, m), c1 = min(c0 + per, m);
    uint32_t sum = 0;
    for (uint32_t i = c0; i < c1; ++i) {
        const SputRec rec = P.squeue[(uint32_t)s_key[i]];
        sum += rec.n;
        atomicAdd(&s_el[rec.meta & 1u], rec.n);
    }
    const int lane = (int)(tid & 31u), w = (int)(tid >> 5);
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t v = s_wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += u;
        }
        s_wsum[lane] = v;                            // inclusive warp totals
    }
    __syncthreads();
    const uint32_t total = s_wsum[SPUT_THREADS / 32 - 1];
    uint32_t off = (w > 0 ? s_wsum[w - 1] : 0u) + incl - sum;
    if (tid == 0) {
        const unsigned long long base = atomicAdd(&st->n_slots, (unsigned long long)total);
        s_ok = base + total <= P.capacity ? 1u : 0u;
        if (!s_ok) set_error(st, ERR_CAPACITY);
        s_base = base;
        RunState& rs = P.rs[r];
        s_id0 = rs.id_next;
        if ((unsigned long long)rs.id_next + total > 0xFFFFFFFFull) set_error(st, ERR_IDS);
        rs.id_next += total;
        if (s_el[0]) rs.ctr[C_SPUT_C] += s_el[0];
        if (s_el[1]) rs.ctr[C_SPUT_A] += s_el[1];
    }
    __syncthreads();
    if (!s_ok) return;
    const RunInfo& RI = P.runs[r];
    uint32_t fb = 0;
    for (uint32_t i = c0; i < c1; ++i) {
        const SputRec rec = P.squeue[(uint32_t)s_key[i]];
        const uint32_t el = rec.meta & 1u;
        const int iz = el == 0u ? 0 : RI.nz - 1;
        const float pz = el == 0u ? 0.0f : 0x1.fffffep-1f;
        const uint32_t gcell = RI.cell_base + (uint32_t)iz * (uint32_t)RI.nr + rec.ir;
        for (uint32_t j = 0; j < rec.n; ++j, ++off) {
            Stream sp(rec.id, st->step, sid_sput_atom(j), RI.seed, RI.run);
            const float U1 = sp.u01(), U2 = sp.u01();
            const float vn = P.sput_vth * rayleigh(ray, U1);
            const float sv = P.sput_vth * rayleigh(ray, U2);
            float cp, sn;
            azimuth(sp, cp, sn, fb);
            // a tail slot after those in use: the atom joins this step's sort as a mover
            const unsigned long long slot = s_base + off;
            M.key[slot] = make_key(SP_CU, gcell);
            M.pz[slot] = pz;
            M.pr[slot] = rec.pr;
            M.vz[slot] = el == 0u ? vn : -vn;
            M.vr[slot] = sv * cp;
            M.vt[slot] = sv * sn;
            M.id[slot] = s_id0 + off;
            atomicOr(&mm[slot >> 5], 1u << (slot & 31u));
            atomicAdd(&in_cnt[(uint32_t)SP_CU * P.ncell + gcell], 1u);
        }
    }
    if (fb) atomicAdd(&P.rs[r].ctr[C_ISOFB], (unsigned long long)fb);
}

cudaError_t collide_setup() {
    cudaError_t e = cudaFuncSetAttribute(k_rank_tables<RT_THREADS, RANK_BLOCK_MAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RT_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_rank_tables<RT_MID_THREADS, RANK_MID_MAX>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RT_MID_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sputter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SPUT_SMEM);
    return e;
}
void launch_ncand(const uint32_t* cnt, const float* ck, uint4* nc, uint4* nc2, uint32_t* cand, uint32_t* active,
                  uint32_t* mid, uint32_t* big, DevState* st, const KParams& P, int grid, cudaStream_t s) {
    if (P.charge_max >= 3 || P.heavy_coll || P.coulomb)
        k_ncand<true><<<grid, 256, 0, s>>>(cnt, ck, nc, nc2, cand, active, mid, big, st, P);
    else
        k_ncand<false><<<grid, 256, 0, s>>>(cnt, ck, nc, nc2, cand, active, mid, big, st, P);
}
void launch_collide(const Particles& A, const Particles& B, const uint32_t* off, const uint32_t* cnt, const uint4* nc,
                    const uint4* nc2,
                    const uint32_t* cand_off, const uint32_t* active, const uint32_t* mid, const uint32_t* big,
                    DevState* st, long long* rho_e, long long* rho_h, const float* xsE, const float* xs,
                    const double* cw, const KParams& P, const CollConsts& cc, uint32_t nbins, int sms, int grid,
                    cudaStream_t s) {
    const RankScratch S{B.key, reinterpret_cast<uint32_t*>(B.pz), reinterpret_cast<uint32_t*>(B.pr),
                        reinterpret_cast<uint32_t*>(B.vz), B.id};
    k_rank_tables<RT_MID_THREADS, RANK_MID_MAX><<<sms * RT_MID_BLOCKS_PER_SM, RT_MID_THREADS, RT_MID_SMEM, s>>>(
        A.id, S, off, cnt, mid, &st->n_mid, rank_queue_max(P.capacity, RANK_WARP_MAX), P.ncell, st);
    k_rank_tables<RT_THREADS, RANK_BLOCK_MAX><<<sms, RT_THREADS, RT_SMEM, s>>>(
        A.id, S, off, cnt, big, &st->n_big, rank_queue_max(P.capacity, RANK_MID_MAX), P.ncell, st);
    if (P.charge_max >= 3 || P.heavy_coll || P.coulomb)
        k_collide<true><<<grid, 128, 0, s>>>(A, S, off, cnt, nc, nc2, cand_off, active, st, rho_e, rho_h, xsE, xs, cw, P,
                                             cc, nbins);
    else
        k_collide<false><<<grid, 128, 0, s>>>(A, S, off, cnt, nc, nc2, cand_off, active, st, rho_e, rho_h, xsE, xs, cw, P,
                                              cc, nbins);
}
void launch_coulomb(const Particles& A, const Particles& B, const uint32_t* off, const uint32_t* cnt, DevState* st,
                    const KParams& P, const CollConsts& cc, const double* cw, int sms, cudaStream_t s) {
    const RankScratch S{B.key, reinterpret_cast<uint32_t*>(B.pz), reinterpret_cast<uint32_t*>(B.pr),
                        reinterpret_cast<uint32_t*>(B.vz), B.id};
    // one wave of resident blocks, grid-stride over the cells
    k_coulomb<<<sms * 6, 32 * COUL_WARPS, 0, s>>>(A, S, off, cnt, st, P, cc, cw);
}
void launch_finalize(const uint32_t* off, uint32_t nbins, const uint32_t* cand_off, DevState* st, const KParams& P,
                     const RunCircuit* circ, double dt, int circuit, cudaStream_t s) {
    k_finalize<<<1, 256, 0, s>>>(off, nbins, cand_off, st, P, circ, dt, circuit);
}
void launch_sputter(const Particles& M, uint32_t* mm, DevState* st, const KParams& P, const float* ray,
                    uint32_t* in_cnt, cudaStream_t s) {
    k_sputter<<<P.nruns, SPUT_THREADS, SPUT_SMEM, s>>>(M, mm, st, P, ray, in_cnt);
}

void launch_inject(Particles A, const float2* E, DevState* st, const KParams& P, const InjectConsts* ic,
                   const float* ray, cudaStream_t s) {
    k_inject<<<P.nruns, 256, 0, s>>>(A, E, st, P, ic, ray);
}

}  // namespace pd
