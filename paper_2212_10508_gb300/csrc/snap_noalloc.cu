// snap_energy_forces_noalloc: SNAP energies and forces with no device allocation at call time.
//
// Who needs it: callers that may not call cudaMalloc while they run -- a host application
// whose device memory is owned by its own pool or allocator, code running inside a region
// where an allocation would synchronise the device or is forbidden (a tight time-stepping
// loop, a real-time or latency-bounded controller), or a plugin host that hands the library a
// fixed memory budget.  The regular snap_energy_forces grows the context's scratch with
// cudaMalloc on the first call of a new size; this variant takes its scratch from one
// fixed-size array compiled into the library instead.
//
// The array below (PMD_NOALLOC_SCRATCH_BYTES = 16 MiB) belongs to this file's CUDA module.
// With lazy module loading (the CUDA default) a module's memory is reserved when the module
// is first used on a device, so pmd_snap_create loads it on its device by asking for the
// array's address; from then on the device holds the array until the process exits and the
// entry point itself allocates nothing.  Host code cannot use the array's name as a device
// address: every call asks the runtime for the address in the current context (cheap once the
// module is loaded, and never stale after the context is re-created).  Every call on a device
// shares the array and leaves its contents behind: two calls whose kernels overlap on the GPU
// (different streams without ordering) race on it.  No part of the scratch has to start at
// zero: the kernels write every entry they later read.
#include "pmd_internal.h"

namespace pmd {

void snap_scratch_sizes(const pmd_snap* s, long na, bool want_B, size_t sz[6]);
int snap_compute_scratch(pmd_snap* s, int nbatch, int n, const double box[3], const double* pos, const double* beta,
                         double* energy, double* forces, double* sumB, const SnapScratch& sc, cudaStream_t st);

static __device__ __align__(256) unsigned char g_snap_noalloc_scratch[PMD_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array in the current context; the first request on a device
// loads this module there (pmd_snap_create makes that request).
int noalloc_scratch_address(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_snap_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
    *out = p;
    return PMD_OK;
}

}  // namespace pmd

using namespace pmd;

extern "C" int snap_energy_forces_noalloc(pmd_snap* s, int nbatch, int natoms, const double box[3],
                                          const double* pos, const double* beta, double* energy, double* forces,
                                          double* sumB, pmd_stream_t stream) {
    if (!s) return fail(PMD_EINVAL, "snap_energy_forces_noalloc: NULL context");
    if (nbatch < 0 || natoms < 1) return fail(PMD_EINVAL, "snap_energy_forces_noalloc: need nbatch >= 0, natoms >= 1");
    int rc = check_box(box, s->p.rcut);
    if (rc) return rc;
    if (nbatch == 0) return PMD_OK;
    if (!pos || !beta) return fail(PMD_EINVAL, "snap_energy_forces_noalloc: pos and beta are required");
    const long na = (long)nbatch * natoms;
    size_t sz[6];
    snap_scratch_sizes(s, na, energy || sumB, sz);
    size_t off[6], total = 0;
    for (int k = 0; k < 6; ++k) {
        off[k] = total;
        total += (sz[k] + 255) / 256 * 256;
    }
    if (total > (size_t)PMD_NOALLOC_SCRATCH_BYTES)
        return fail(PMD_EUNSUPPORTED, "snap_energy_forces_noalloc: nbatch*natoms = " + std::to_string(na) +
                                          " needs " + std::to_string(total) + " bytes of scratch; the static array holds " +
                                          std::to_string((size_t)PMD_NOALLOC_SCRATCH_BYTES) + " bytes");
    void* base = nullptr;
    if ((rc = noalloc_scratch_address(&base))) return rc;
    unsigned char* b = static_cast<unsigned char*>(base);
    SnapScratch sc{reinterpret_cast<int*>(b + off[0]), reinterpret_cast<int*>(b + off[1]), b + off[2],
                   reinterpret_cast<float4*>(b + off[3]), sz[4] ? b + off[4] : nullptr,
                   sz[5] ? reinterpret_cast<double*>(b + off[5]) : nullptr};
    return snap_compute_scratch(s, nbatch, natoms, box, pos, beta, energy, forces, sumB, sc, (cudaStream_t)stream);
}
