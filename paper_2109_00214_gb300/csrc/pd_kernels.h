// pd_kernels.h -- host-side launchers of the library's kernels.
#pragma once
#include "pd_internal.cuh"

namespace pd {

constexpr int SCAN_THREADS = 256;
constexpr uint32_t SCAN_TILE = SCAN_THREADS * 8;   // elements per scan block

inline uint32_t scan_padded(uint64_t n) { return (uint32_t)((n + SCAN_TILE - 1) / SCAN_TILE * SCAN_TILE); }

// external circuit of one run
struct RunCircuit {
    double V0, R_ohm, C_farad;
};

// cathode injection constants of one run (ntip = 0: emission off)
struct InjectConsts {
    int ntip;                 // tip cells (r index 0 .. ntip-1)
    double area[64];          // emitting area of each tip cell (m^2)
    float lo[64], hi[64];     // radial extent of each tip cell in cell units
    double dt, weight, beta, work, ratio;
    float vth;                // thermal speed of the neutrals
};

// push + deposit + mover bookkeeping (see pd_stream.cu)
void launch_push(const Particles& A, const float2* E, long long* rho_e, long long* rho_h, uint32_t* out_cnt,
                 uint32_t* in_cnt, uint32_t* mv, uint32_t* mm, const Particles& M, DevState* st, const KParams& P,
                 int grid, cudaStream_t s);
// the sort after the push (see pd_stream.cu)
struct SortArgs {
    Particles A, B;                  // the particles; B: scratch of a re-layout
    Particles M;                     // movers, at their slots' indices
    uint32_t *mv, *mm;               // vacated slots; slots with a mover record
    uint32_t *off, *off2;            // bin starts (nbins_pad + 1 entries), the next layout / scratch
    uint32_t *cnt, *out_cnt, *in_cnt;  // live count, movers out, movers in (cursor) per bin
    uint32_t* cap;                   // re-layout: heavy bin capacities (scan input)
    uint32_t* act;                   // movers in + out per heavy bin since the last layout
    int* net;                        // movers in - out per heavy bin since the last layout
    uint4* bigq;                     // long heavy bins with holes
    uint32_t bigq_cap;
    uint32_t* ovq;                   // heavy bins that outgrew their slots (OVQ_CAP entries)
    uint32_t* ovbits;                // the same as a bit per bin (nbins / 32 + 1 words)
    uint32_t* partial;               // scan partials
    uint32_t nbins, nbins_pad, ncell_pad;
    uint64_t slots;                  // physical slots of the particle arrays
};
// heavy bins: counts, holes closed, slots borrowed by full bins (three launches)
void launch_sort(const SortArgs& a, DevState* st, const KParams& P, int sms, cudaStream_t s);
// a new layout of the heavy bins when one overflowed (every kernel returns at
// once otherwise; ten launches).  first: no particle is in a bin yet (the
// first step after the loads), so the layout is written into A directly
void launch_relayout(const SortArgs& a, DevState* st, const KParams& P, int grid_bins, int grid_slots,
                     cudaStream_t s, bool first);
// the electron bins packed after the heavy bins, then every mover into its
// bin (six launches)
void launch_insert(const SortArgs& a, DevState* st, const KParams& P, int grid_dense, cudaStream_t s);
// heavy bins that may borrow slots from their neighbours in one step (more
// lay the bins out anew)
constexpr uint32_t OVQ_CAP = 65536;
// queue entries that always suffice for bins longer than the warp-compaction
// threshold (they hold disjoint slots)
inline uint32_t bigq_max(uint64_t slots) { return (uint32_t)(slots / 96 + 16); }
void launch_deposit(const Particles& A, long long* rho_e, long long* rho_h, DevState* st, const KParams& P,
                    int grid, cudaStream_t s);
// exclusive scan of n_padded (multiple of SCAN_TILE) u32; out has n_padded + 1
// entries, out[n_padded] = total; partial needs n_padded / SCAN_TILE + 1 entries
// (cond: when not null, the scan runs only if *cond is nonzero)
void launch_scan(const uint32_t* in, uint32_t* out, uint32_t* partial, uint32_t n_padded, cudaStream_t s,
                 const uint32_t* cond = nullptr);
// the same over the population counts of the input words
void launch_scan_popc(const uint32_t* in, uint32_t* out, uint32_t* partial, uint32_t n_padded, cudaStream_t s);
// diagnostics of one run
// live particles of every run and species, out[run * NSP + species] (zeroed by the caller)
void launch_species_count_all(const Particles& A, DevState* st, const KParams& P, unsigned long long* out, int grid,
                              cudaStream_t s);
void launch_density(const Particles& A, DevState* st, const KParams& P, int run, int species, long long* acc,
                    int grid, cudaStream_t s);
void launch_spectrum(const Particles& A, DevState* st, const KParams& P, int run, int species, double lo, double hi,
                     int nbins, unsigned long long* hist, int grid, cudaStream_t s);

// device-array load: keys and ids of n new particles of one run; *bad set on a bad input
void launch_pack_keys(const uint8_t* sp, const int32_t* iz, const int32_t* ir, const float* pz, const float* pr,
                      int64_t n, int nz, int nr, uint32_t cell_base, uint32_t id0, uint32_t sp_max, uint32_t* key,
                      uint32_t* id, unsigned int* bad, int grid, cudaStream_t s);

// collisions.  The rank table of an id list of more than RANK_WARP_MAX ids
// (beyond a warp's register cache) that the candidates of an active cell use
// is built before k_collide, by a block of its own: lists up to RANK_MID_MAX
// ids by the mid-size kernel, longer ones by the large one.  k_ncand queues
// them in `mid` and `big`; rank_queue_max(cap, len) entries always suffice
// for lists longer than len (the lists hold disjoint particles).
constexpr uint32_t RANK_WARP_MAX = 256;
constexpr uint32_t RANK_MID_MAX = 2048;
__host__ __device__ inline uint32_t rank_queue_max(uint64_t cap, uint32_t len) { return (uint32_t)(cap / (len + 1) + 4); }
// shared-memory attribute of the rank-table kernels (once per process and device)
cudaError_t collide_setup();
// nc: candidates of classes 0, 1, 5, 6; nc2: classes 2, 3, 4 (written with charge_max >= 3)
void launch_ncand(const uint32_t* cnt, const float* ck, uint4* nc, uint4* nc2, uint32_t* cand, uint32_t* active,
                  uint32_t* mid, uint32_t* big, DevState* st, const KParams& P, int grid, cudaStream_t s);
// B: the other particle buffer, used as scratch (free outside a re-layout);
// off / cnt: bin starts and live counts.  The two rank-table kernels, then
// k_collide (three launches)
void launch_collide(const Particles& A, const Particles& B, const uint32_t* off, const uint32_t* cnt, const uint4* nc,
                    const uint4* nc2,
                    const uint32_t* cand_off, const uint32_t* active, const uint32_t* mid, const uint32_t* big,
// cw: W dt_coll / V_cell per row (Coulomb pairs)
                    DevState* st, long long* rho_e, long long* rho_h, const float* xsE, const float* xs,
                    const double* cw, const KParams& P, const CollConsts& cc, uint32_t nbins, int sms, int grid,
                    cudaStream_t s);
// Coulomb pairs (after launch_collide; one launch)
void launch_coulomb(const Particles& A, const Particles& B, const uint32_t* off, const uint32_t* cnt, DevState* st,
                    const KParams& P, const CollConsts& cc, const double* cw, int sms, cudaStream_t s);
// ion-impact sputtering after the push (one block per run): the atoms go to
// the mover records M (mask mm) of tail slots; in_cnt: the movers-into-bin
// counts of the sort
void launch_sputter(const Particles& M, uint32_t* mm, DevState* st, const KParams& P, const float* ray,
                    uint32_t* in_cnt, cudaStream_t s);
void launch_finalize(const uint32_t* off, uint32_t nbins, const uint32_t* cand_off, DevState* st, const KParams& P,
                     const RunCircuit* circ, double dt, int circuit, cudaStream_t s);

// cathode injection, one block per run
void launch_inject(Particles A, const float2* E, DevState* st, const KParams& P, const InjectConsts* ic,
                   const float* ray, cudaStream_t s);

}  // namespace pd
