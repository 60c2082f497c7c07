// pd_noalloc.cu -- energy histogram of raw device particle arrays with no
// allocation at all.
//
// Who this is for: callers that hold particle arrays in device memory (for
// example, state restored by another framework, or buffers exported by a
// tool) and that cannot allocate device memory to get a diagnostic.  Some
// cannot call cudaMalloc because device memory belongs to someone else's
// allocator or budget.  Others run where an allocation is not allowed: an
// allocation also synchronises the device and would stall the simulation.
// pd_get_energy_spectrum needs a pd_sim and its workspace.  This entry point
// needs neither.  Its histogram scratch is a fixed array in the library's
// own device memory (PD_SPECTRUM_STATIC_MAX_BINS counters, 32 KiB), which
// every GPU that loads the library keeps until the process exits.
//
// Compiled with -fmad=false, like pd_particles.cu, so each energy is rounded
// operation by operation exactly as the pd_get_energy_spectrum kernel does
// it, and the two give the same bins.
#include <cstdio>
#include <mutex>

#include "pd.h"
#include "pd_internal.cuh"

namespace pd {

// The scratch: one histogram, shared by every call on a device.
static __device__ __align__(256) unsigned long long g_spectrum_scratch[PD_SPECTRUM_STATIC_MAX_BINS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long* g_scratch_ptr[kMaxDevices] = {};   // device address of the array, per device

// Host code cannot use the array's name as a device address.  Ask the
// runtime for it once per device (the device must be current) and remember
// it for the life of the process (a cudaDeviceReset in the process would
// leave the remembered address stale).
cudaError_t scratch_for_current_device(unsigned long long** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_spectrum_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (unsigned long long*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

__global__ void k_spectrum_raw(const uint32_t* __restrict__ key, const float* __restrict__ vz,
                               const float* __restrict__ vr, const float* __restrict__ vt, long long n,
                               uint32_t species, double mass, double lo, double hi, int nbins,
                               unsigned long long* hist) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t k = key[i];
        if (k == DEAD || key_species(k) != species) continue;
        const double a = vz[i], b = vr[i], c = vt[i];
        const double v2 = a * a + b * b + c * c;
        const double e = 0.5 * mass * v2 / 1.602176634e-19;
        if (e < lo || e >= hi) continue;
        int bin = (int)((e - lo) / (hi - lo) * nbins);
        if (bin >= nbins) bin = nbins - 1;
        atomicAdd(&hist[bin], 1ull);
    }
}

}  // namespace
}  // namespace pd

extern "C" pd_status pd_energy_spectrum_static(const uint32_t* key, const float* vz, const float* vr,
                                               const float* vt, int64_t n, int species, double e_lo_eV,
                                               double e_hi_eV, int nbins, void* cuda_stream, uint64_t* out) {
    using namespace pd;
    if (nbins < 1 || nbins > PD_SPECTRUM_STATIC_MAX_BINS) {
        std::fprintf(stderr, "pd_energy_spectrum_static: nbins = %d is outside 1..%d\n", nbins,
                     PD_SPECTRUM_STATIC_MAX_BINS);
        return PD_ERR_ARG;
    }
    if (n < 0 || species < 0 || species >= NSP || !(e_hi_eV > e_lo_eV) || !out) return PD_ERR_ARG;
    if (n > 0 && (!key || !vz || !vr || !vt)) return PD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the scratch address is the current device's: the stream must be on it
    int sdev = -1, cur = -1;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess || cudaGetDevice(&cur) != cudaSuccess) return PD_ERR_CUDA;
    if (sdev != cur) {
        std::fprintf(stderr, "pd_energy_spectrum_static: the stream is on device %d, the current device is %d\n", sdev,
                     cur);
        return PD_ERR_ARG;
    }
    unsigned long long* hist = nullptr;
    if (scratch_for_current_device(&hist) != cudaSuccess) return PD_ERR_CUDA;
    // the array keeps the previous call's counts: clear the bins used here
    if (cudaMemsetAsync(hist, 0, (size_t)nbins * sizeof(unsigned long long), s) != cudaSuccess) return PD_ERR_CUDA;
    if (n > 0) {
        const double mass = species_mass_kg(species);     // the masses pd_get_energy_spectrum uses
        long long blocks = (n + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        k_spectrum_raw<<<(unsigned)blocks, 256, 0, s>>>(key, vz, vr, vt, (long long)n, (uint32_t)species, mass,
                                                        e_lo_eV, e_hi_eV, nbins, hist);
        if (cudaGetLastError() != cudaSuccess) return PD_ERR_CUDA;
    }
    if (cudaMemcpyAsync(out, hist, (size_t)nbins * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return PD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PD_ERR_CUDA;
    return PD_OK;
}

extern "C" int pd_spectrum_static_max_bins(void) { return PD_SPECTRUM_STATIC_MAX_BINS; }
