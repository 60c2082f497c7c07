// pd_warp.cuh -- warp-level aggregation helpers shared by the particle kernels.
#pragma once
#include "pd_internal.cuh"

namespace pd {

constexpr unsigned FULL_MASK = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum_ull(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// histogram increment with one atomic per distinct bin in the warp
__device__ __forceinline__ void warp_count(uint32_t* count, uint32_t bin, bool on) {
    const unsigned m = __ballot_sync(FULL_MASK, on);
    if (!on) return;
    const unsigned g = __match_any_sync(m, bin);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(g) - 1)) atomicAdd(&count[bin], (uint32_t)__popc(g));
}

// Fixed-point CIC deposit, Eq. (9)-(10): w = rn(f * 2^16) per axis, corner
// weights (2^16 - w_z)(2^16 - w_r), w_z (2^16 - w_r), (2^16 - w_z) w_r, w_z w_r
// (they sum to 2^32).  Lanes holding the same key (species and cell) are
// summed first: each weight is split in 16-bit halves so the warp sums fit in
// 32 bits, then one 64-bit atomic per node and group.  (iz, ir) are local to
// the run RI.
__device__ __forceinline__ void warp_deposit(long long* rho, const RunInfo& RI, int geom, uint32_t key, int iz, int ir,
                                             float pz, float pr, int zq, bool on) {
    const unsigned m = __ballot_sync(FULL_MASK, on);
    if (!on) return;
    const unsigned g = __match_any_sync(m, key);
    const uint32_t wz = __float2uint_rn(pz * 65536.0f);
    const uint32_t wr = __float2uint_rn(pr * 65536.0f);
    const unsigned long long az = 65536u - wz, ar = 65536u - wr;
    const unsigned long long W[4] = {az * ar, (unsigned long long)wz * ar, az * (unsigned long long)wr,
                                     (unsigned long long)wz * wr};
    const bool leader = (threadIdx.x & 31) == (unsigned)(__ffs(g) - 1);
    const uint32_t nodes[4] = {node_of(RI, geom, iz, ir), node_of(RI, geom, iz + 1, ir), node_of(RI, geom, iz, ir + 1),
                               node_of(RI, geom, iz + 1, ir + 1)};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t hi = __reduce_add_sync(g, (uint32_t)(W[k] >> 16));
        const uint32_t lo = __reduce_add_sync(g, (uint32_t)(W[k] & 0xFFFFu));
        if (leader) {
            const long long s = (long long)(((unsigned long long)hi << 16) + lo) * zq;
            atomicAdd((unsigned long long*)&rho[nodes[k]], (unsigned long long)s);
        }
    }
}

}  // namespace pd
