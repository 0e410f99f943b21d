// Internal declarations of the pmd library (host side): contexts, tables, error helpers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pmd.h"
#include "status_bits.h"

namespace pmd {

// ---- errors ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t err, const char* what);

#define PMD_CUDA_TRY(call)                                         \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::pmd::cuda_fail(_e, #call); \
    } while (0)

int status_to_code(int bits);

// PMD_OK if every box edge is finite and exceeds 2 rc, else PMD_EINVAL with a message.
int check_box(const double box[3], double rc);

// ---- device buffers --------------------------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    int ensure(size_t need);   // grow (never shrinks); returns PMD_OK or an error code
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// ---- SNAP tables -----------------------------------------------------------------------
// Half layout of U and Y: for each level tj (= 2j), rows p = 0..tj (p = j + m'),
// columns q = qlo(tj)..tj (q = j + m, m >= 0), qlo = (tj + 1) / 2, row-major.
// Full layout: rows p = 0..tj, columns q = 0..tj, row-major, levels concatenated.
inline int qlo(int tj) { return (tj + 1) / 2; }
inline int ncol_half(int tj) { return tj + 1 - qlo(tj); }
inline int uoff_full(int tj) { return tj * (tj + 1) * (2 * tj + 1) / 6; }

struct SnapHostTables {
    int twojmax = 0;
    int nB = 0;                       // bispectrum components
    int nhalf = 0, nfull = 0;         // element counts of the half and full layouts
    std::vector<int> tri;             // [nB][3] (2j1, 2j2, 2j), j2 <= j1 <= j
    // U half elements: recursion and force-pass metadata
    std::vector<int> hoff;            // [twojmax+2] offsets of each level in the half layout
    // contraction blocks (ta >= tb, tj): Z^j_{ab} feeds Y^j with coefficient beta_eff(block)
    std::vector<int> blk_ta, blk_tb, blk_tj, blk_cgoff;
    std::vector<double> cg;           // per block [(ta+1)][(tb+1)]: <a m1 b m2 | J m1+m2>
    std::vector<int> beff_ptr;        // CSR over blocks: contributions (t, coef)
    std::vector<int> beff_t;
    std::vector<double> beff_c;
    // Y jobs in lockstep rounds: [nrounds][32] int4 records, every round one sub-block size tb
    std::vector<int> jobs;            // [nrounds * 32][4]
    std::vector<unsigned char> round_tb;
    int nrounds = 0;
    double total_terms = 0;           // Clebsch-Gordan terms per atom (algorithmic, unpadded)
    double padded_terms = 0;          // term slots executed (lockstep padding included)
    // batched Y phase (FP32, lane = atom): int4 jobs (row, block) grouped by owning warp
    std::vector<int> sb_jobs;         // [njobs][4]
    std::vector<int> sb_rows;         // [nrows][2] job range of each (stage, row), stages concatenated
    std::vector<int> sb_sptr;         // [nstages + 1] row ranges of the stages
    std::vector<int> sb_groups;       // [ngroups][2] (first row, count): equal-width rows, 2 or 4 per group
    std::vector<int> sb_gptr;         // [2][nstages][2] group ranges [begin, end) per stage (R = 2, then R = 4)
    std::vector<float> sb_coef;       // per-job Clebsch-Gordan weights (column, then row)
    double sb_load_max = 0, sb_load_avg = 0;
    // bispectrum jobs (energy path): per triple t the block id of (j1, j2, j)
    std::vector<int> tri_blk;
};
int build_snap_tables(int twojmax, SnapHostTables* T);

// device scratch of one snap_energy_forces call
struct SnapScratch {
    int* nbr;       // [na][PMD_MAX_NEIGHBORS]
    int* nnb;       // [na]
    void* dedr;     // [na][PMD_MAX_NEIGHBORS][3] reals
    float4* qf;     // [na]
    void* utot;     // [na][nfull] complex reals (energy path)
    double* B;      // [na][nB] (energy path)
};

}  // namespace pmd

// ---- contexts -------------------------------------------------------------------------
struct pmd_snap {
    pmd_snap_params p;
    pmd::SnapHostTables T;
    int device = 0;
    // device copies of the tables
    pmd::DevBuf d_cg;        // CG values (precision dependent)
    pmd::DevBuf d_blk;       // int4 per block {ta, tb, tj, cgoff}
    pmd::DevBuf d_beffptr, d_befft, d_beffc;
    pmd::DevBuf d_jobs;      // int4 jobs [nrounds][32]
    pmd::DevBuf d_roundtb;   // uint8 [nrounds]
    pmd::DevBuf d_triblk;    // int4 per triple {blk, ta, tb, tj}
    pmd::DevBuf d_sbjobs;    // int4 jobs of the batched Y phase
    pmd::DevBuf d_sbrows;    // int2 job range per (stage, row)
    pmd::DevBuf d_sbsptr;    // int [nstages + 1]
    pmd::DevBuf d_sbcoef;    // float per-job Clebsch-Gordan weights
    pmd::DevBuf d_sbgroups;  // int2 row groups for multi-row warps
    pmd::DevBuf d_sbgptr;    // int [2][nstages][2]
    // scratch
    pmd::DevBuf s_nbr, s_nnb, s_dedr, s_qf, s_utot, s_B, s_status;
    int cap_atoms = 0;
};

struct pmd_engine {
    pmd_engine_params p;
    pmd_snap* snap = nullptr;        // owned
    pmd::DevBuf beta;                // [1+nB] FP64
    pmd_snap* csnap = nullptr;       // SNAP coarse potential (PMD_COARSE_SNAP), owned
    pmd::DevBuf cbeta;               // its coefficients [1+nB] FP64
    pmd::DevBuf status;              // int status word + barrier words
    pmd::DevBuf s_nbr, s_nnb, s_dedr, s_qf, s_vh, s_order, s_Ls, s_result;
    pmd::DevBuf s_noise;             // Gaussian increments of a parareal_correct window
    pmd::DevBuf s_selftest;          // words of pmd_engine_selftest_waits
    pmd::DevBuf s_flow;              // FP32 fine path: item counter, abort word, per-member phase counters
    pmd::DevBuf s_gstep;             // Gaussian increments of one fine sub-step [item][3] (FP32 path)
    pmd::DevBuf s_pos;               // reverse neighbour slots [member][j][k] (uint8), natoms <= PMD_POS_TABLE_MAX_ATOMS
    int cap_batch = 0;
    int device = 0;
    int num_sms = 0;
    void* pinned = nullptr;          // small pinned host buffer for parareal_correct results
    int profile = 0;                 // record events around the persistent FINE kernel
    pmd_fine_tuning tune = {16, 8, 8, -1, 16};   // run-time shape of the batched FP32 kernel (autotuned)
    int prof_recorded = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

struct pmd_adaptive;  // defined in adaptive.cpp

// systems up to this size keep a table of reverse neighbour slots (natoms^2 bytes per member)
constexpr int PMD_POS_TABLE_MAX_ATOMS = 2048;
