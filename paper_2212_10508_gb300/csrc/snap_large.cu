// snap_energy_forces for the band limits 2J = 10, 12 and 14 (14: the paper's SNAP-205), FP64,
// one warp per atom: the kernels of snap_launch.cuh instantiated in a translation unit of their
// own (their unrolled recursions over 271-652 half elements take most of the library's compile
// time, which then overlaps with the other units).
#include "snap_launch.cuh"

namespace pmd {

int snap_launch_large(pmd_snap* s, int nbatch, int n, const double box[3], const double* pos, const double* beta,
                      double* energy, double* forces, double* sumB, const SnapScratch& sc, cudaStream_t st) {
    switch (s->p.twojmax) {
        case 10: return launch_snap<double, 10>(s, nbatch, n, box, pos, beta, energy, forces, sumB, sc, st);
        case 12: return launch_snap<double, 12>(s, nbatch, n, box, pos, beta, energy, forces, sumB, sc, st);
        case 14: return launch_snap<double, 14>(s, nbatch, n, box, pos, beta, energy, forces, sumB, sc, st);
    }
    return fail(PMD_EUNSUPPORTED, "snap_launch_large: twojmax must be 10, 12 or 14");
}

}  // namespace pmd
