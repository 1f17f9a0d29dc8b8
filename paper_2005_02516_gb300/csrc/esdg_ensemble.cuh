// Declarations of the ensemble path (esdg_ensemble_impl.cuh): the tile table
// entry of a member, the warp budget, and the host wrappers.
#pragma once

#include "esdg_stage2.cuh"

namespace esdg {

// ---- ensembles: several independent problems in one persistent launch --------
// Tile table: problem i owns the global batches [batch_begin, batch_begin +
// nbatch); every batch is EPW = 4 consecutive elements of that problem.
struct EnsembleMember {
    StageParams<float> p;   // all fields but ut_in/ut_out/rkA/rkB (set per launch)
    const float* ops2;      // operators of the member's degree (k_stage2 layout)
    float* ut[2];           // entropy-projected values, ping-pong
    int N;                  // degree 1..5 (all members share one volume rule)
    int batch_begin, nbatch;
};

// Warps per block of the ensemble kernel (96 registers a thread).  Its
// per-degree batch bodies are separate (not inlined) functions, so each gets
// the register budget alone rather than the union of every degree's paths:
// 20 warps then run without spills, 7% faster than 16 warps at 128 registers
// with the bodies inlined (config 4: 9.45 against 8.80 GDOF-stage/s).
constexpr int ENSEMBLE_MAX_WARPS = 20;
// With degree-5 members (whose body needs 128 registers, as in k_stage2) the
// instantiation that carries the degree-5 path runs 16 warps.
constexpr int ensemble_max_warps(int nmax) { return nmax >= 5 ? 16 : ENSEMBLE_MAX_WARPS; }

// Host wrappers of the ensemble kernel (esdg_ensemble_impl.cuh), one
// instantiation per volume rule RULE (0 collapsed, 1 symmetric) in its own
// translation unit: shared-memory attribute and launch, for members of degree
// at most nmax (4 or 5).
template <int RULE>
cudaError_t ensemble_smem_attr(int nmax, size_t smem);
template <int RULE>
cudaError_t launch_ensemble(int nmax, int grid, int block, size_t smem, cudaStream_t s, const EnsembleMember* mem,
                            int nmem, int total_batches, int which, double rkA, double rkB, int4 ops_lo, int ops_hi,
                            int ops_end, int slab);

}  // namespace esdg
