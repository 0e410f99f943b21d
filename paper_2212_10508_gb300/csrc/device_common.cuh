// Device helpers shared by the pmd kernels: complex arithmetic, counter-based noise,
// status reporting and a bounded grid barrier for persistent cooperative kernels.
#pragma once

#include <cuda_runtime.h>
#include <cuda/atomic>
#include <stdint.h>

#include "status_bits.h"

namespace pmd {

constexpr double KB = 8.617333262e-5;        // eV/K
constexpr double FTOA = 9648.533215665;      // 1 eV/(Angstrom u) in Angstrom/ps^2
constexpr double PI = 3.14159265358979323846;

template <typename real>
struct cplx {
    real re, im;
};
template <typename real>
__device__ __forceinline__ cplx<real> cmul(cplx<real> a, cplx<real> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <typename real>
__device__ __forceinline__ cplx<real> cmulc(cplx<real> a, cplx<real> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

// ---- status -----------------------------------------------------------------------------
__device__ __forceinline__ void flag(int* status, int bits) {
    if (status) atomicOr(status, bits);
}

// ---- noise: Philox4x32-10 (Salmon et al., SC'11) + Box-Muller ---------------------------
// Counter (2*atom + blk, l, n_lo, n_hi), key (seed_lo, seed_hi).  Ten rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)), key bumped by the
// Weyl constants between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = __umulhi(m0, c[0]), lo0 = m0 * c[0];
        uint32_t hi1 = __umulhi(m1, c[2]), lo1 = m1 * c[2];
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// Two standard normals from one Philox block: 53-bit uniforms U1 (-> u1 = 1 - U1 in (0,1])
// and u2 in [0,1); (sqrt(-2 ln u1) cos 2 pi u2, sqrt(-2 ln u1) sin 2 pi u2).
__device__ __forceinline__ void box_muller(const uint32_t x[4], double& ga, double& gb) {
    const double two_m53 = 1.0 / 9007199254740992.0;
    double U1 = (double)(((uint64_t)(x[0] >> 5) << 26) | (uint64_t)(x[1] >> 6)) * two_m53;
    double u2 = (double)(((uint64_t)(x[2] >> 5) << 26) | (uint64_t)(x[3] >> 6)) * two_m53;
    double u1 = 1.0 - U1;
    double R = sqrt(-2.0 * log(u1));
    double ang = __dmul_rn(2.0 * PI, u2);
    double s, c;
    sincos(ang, &s, &c);
    ga = R * c;
    gb = R * s;
}

// G_{l,n} of one atom (x, y, z).
__device__ __forceinline__ void normals3(uint64_t seed, int64_t n, int ell, int atom, double g[3]) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint64_t un = (uint64_t)n;
    uint32_t c[4] = {2u * (uint32_t)atom, (uint32_t)ell, (uint32_t)un, (uint32_t)(un >> 32)};
    philox4x32_10(c, k0, k1);
    box_muller(c, g[0], g[1]);
    uint32_t d[4] = {2u * (uint32_t)atom + 1u, (uint32_t)ell, (uint32_t)un, (uint32_t)(un >> 32)};
    philox4x32_10(d, k0, k1);
    double unused;
    box_muller(d, g[2], unused);
}

// ---- bounded grid barrier ---------------------------------------------------------------
// Words: [0] arrival count, [1] generation, [2] abort flag.  All CTAs of a cooperative launch
// call it.  A CTA that waits longer than the spin limit sets the abort flag and the status
// ST_TIMEOUT bit and returns false; every later barrier then returns false at once, so all
// CTAs leave the persistent loop.
struct GridBarrier {
    unsigned int* words;
    unsigned int nblocks;
};

// Spin limit of every cross-CTA wait: about 4 s at ~200 ns per poll, far above any legitimate wait.
constexpr long long WAIT_POLLS = 20000000LL;

// One thread: wait until *ctr >= target, at most `limit` polls.  The abort word ends the wait at
// once (false); running out of polls sets the abort word and the status bit and returns false.
// U: unsigned int or unsigned long long words.
template <typename U>
__device__ __forceinline__ bool bounded_wait_geq(U* ctr, U target, U* abort_word, int* status, int timeout_bit,
                                                 long long limit = WAIT_POLLS) {
    cuda::atomic_ref<U, cuda::thread_scope_device> x(*ctr), ab(*abort_word);
    long long it = 0;
    while (x.load(cuda::memory_order_acquire) < target) {
        if (ab.load(cuda::memory_order_relaxed) != 0) return false;
        if (++it > limit) {
            ab.store(U(1), cuda::memory_order_relaxed);
            flag(status, timeout_bit);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

__device__ __forceinline__ bool grid_sync(GridBarrier gb, int* status, int timeout_bit, long long limit = WAIT_POLLS) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(gb.words[0]);
        cuda::atomic_ref<unsigned int, cuda::thread_scope_device> gen(gb.words[1]);
        cuda::atomic_ref<unsigned int, cuda::thread_scope_device> abrt(gb.words[2]);
        int ok = abrt.load(cuda::memory_order_acquire) == 0;
        if (ok) {
            unsigned int g = gen.load(cuda::memory_order_acquire);
            unsigned int arrived = cnt.fetch_add(1u, cuda::memory_order_acq_rel);
            if (arrived == gb.nblocks - 1) {
                cnt.store(0u, cuda::memory_order_relaxed);
                gen.fetch_add(1u, cuda::memory_order_acq_rel);
            } else {
                long long it = 0;
                while (gen.load(cuda::memory_order_acquire) == g) {
                    if (abrt.load(cuda::memory_order_relaxed) != 0) {
                        ok = 0;
                        break;
                    }
                    if (++it > limit) {
                        abrt.store(1u, cuda::memory_order_relaxed);
                        flag(status, timeout_bit);
                        ok = 0;
                        break;
                    }
                    __nanosleep(100);
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace pmd
