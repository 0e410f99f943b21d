// Langevin sub-steps (Sec. 2, eqs. (2)-(3) and the corrected eqs. (11)-(12) with the
// schedules (13)-(14); option BAOAB), per degree of freedom, FP64.  Every product and sum
// is rounded separately (no fused multiply-add), in the order of the written scheme:
//   v_{l+1/2} = ((v_l + (dt/2 F/m)) - (dt/2 gamma) v_{l-1/2}) + s(C_l) G_l,   q += dt v_{l+1/2}
//   v_{l+1}   = ((v_{l+1/2} + (dt/2 F/m)) - (dt/2 gamma) v_{l+1/2}) + s(C_{l+1}) G_{l+1}
// with s(C) = 1/2 sqrt(2 gamma kT C dt / m).
#pragma once

#include "device_common.cuh"

namespace pmd {

struct LangevinDev {
    double dt, hdt, hdf, hdg;   // dt, dt/2, (dt/2)(FTOA/m), (dt/2) gamma
    double c1, c2;              // BAOAB: exp(-gamma dt), sqrt(kT/m (1 - c1^2))
    double sig[4];              // s(C) for C = 0..3
    int scheme, schedule;
    uint64_t seed;
};

// (selects rather than an indexed load, so that a kernel-parameter copy of L needs no local memory)
__device__ __forceinline__ double sched_sigma(const LangevinDev& L, int ell) {
    if (L.schedule == PMD_SCHED_ROBUST) return ell == 0 ? L.sig[3] : L.sig[1];
    if (L.schedule == PMD_SCHED_L1_SYM) return L.sig[2];
    return L.sig[1];
}

// half kick: base + dt/2 a - dt/2 gamma vdamp + s G
__device__ __forceinline__ double half_kick(const LangevinDev& L, double base, double F, double vdamp, double s,
                                            double G) {
    double t = __dadd_rn(base, __dmul_rn(L.hdf, F));
    t = __dsub_rn(t, __dmul_rn(L.hdg, vdamp));
    return __dadd_rn(t, __dmul_rn(s, G));
}

__device__ __forceinline__ double drift(double q, double dt, double v) { return __dadd_rn(q, __dmul_rn(dt, v)); }

// BAOAB pieces
__device__ __forceinline__ double kick_b(const LangevinDev& L, double v, double F) {
    return __dadd_rn(v, __dmul_rn(L.hdf, F));
}
__device__ __forceinline__ double ou_o(const LangevinDev& L, double v, double G) {
    return __dadd_rn(__dmul_rn(L.c1, v), __dmul_rn(L.c2, G));
}

}  // namespace pmd
