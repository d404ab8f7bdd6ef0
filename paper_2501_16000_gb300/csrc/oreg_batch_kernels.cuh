// Batched stream-collide: one persistent kernel advances many independent
// lattices of any size by one time step, walking a flattened table of warp
// work items (one row segment of one lattice each).
//
// Every lattice keeps its own population memory, geometry, relaxation time
// and equilibrium constants in a device descriptor.  A device-resident global
// step counter g decides, per lattice, whether it is active in this launch
// (g_base <= g < g_end) and at which local time t = t_base + (g - g_base),
// which selects the A-B buffer or the AA parity.  The launches of K steps and
// one counter increment are captured once in a CUDA graph; joining and
// leaving lattices only rewrite the descriptor, item and group tables, so the
// graph is never re-captured.
#pragma once

#include <cuda_runtime.h>

#include "oreg_device.cuh"
#include "oreg_kernels.cuh"
#include "oreg_launch.h"

namespace oreg {

template <typename C> struct BatchDesc {
    void *mem;            // population memory (A-B: two buffers back to back)
    int nx, ny, pitch;
    int eq, coll;
    int lw;               // log2 of the lanes per row segment
    size_t plane;         // elements per plane
    size_t buf_elems;     // elements per population buffer
    long long t_base;     // lattice time when the global step counter was g_base
    long long g_base;     // first global step the lattice takes part in
    long long g_end;      // first global step it no longer takes part in
    int sr;               // stochastic rounding of half formats
    CollConst<C> k;
};

// Work items are grouped on the host by (walls, equilibrium kind, collision,
// parity class): group = ((walls * 3 + eq) * 2 + coll) * 2 + c, with eq the
// kernel's equilibrium kind (guided, polynomial, guided at the local
// temperature) and
// c = (t_base - g_base) & 1 the lattice's fixed offset between its own time
// and the global step, so that at global step g every lattice of class c has
// time parity (g + c) & 1.  Each kernel below handles one (walls, eq, coll)
// and, for the in-place layout, one parity: one item body per kernel keeps
// register use at the single-lattice kernels' level.  groups[0..24] are the
// item offsets of the 24 groups.  A batch launches only the kernels of the
// (walls, eq, coll) combinations its members use (bit ((walls * 3 + eq) * 2
// + coll) of BatchLaunch::combos).
enum { BATCH_AB = 0, BATCH_AA_EVEN = 1, BATCH_AA_ODD = 2 };

// At most 128 threads x 3 blocks per SM (a 170-register cap): the per-lattice
// constants come from the descriptor in global memory rather than the
// parameter bank, and left to itself the compiler keeps them all in registers
// (150-180 for half storage), halving occupancy.  On 512 mixed FP16 lattices
// tighter caps that buy more warps spill and run slower (128 registers: -10%,
// 144: -4%; the kernel uses ~155 at this bound).
constexpr int BATCH_MAX_THREADS = 128;
template <int S, int KIND, int EQ, int COLL, bool WALLS>
__global__ void __launch_bounds__(BATCH_MAX_THREADS, 3)
    k_batch_step(const BatchDesc<typename Storage<S>::C> *__restrict__ descs,
                 const int4 *__restrict__ items, const int *__restrict__ groups,
                 const long long *__restrict__ g_round, int k) {
    using T = typename Storage<S>::T;
    const long long g = *g_round + k;
    constexpr int combo = ((WALLS ? 1 : 0) * 3 + EQ) * 2 + COLL;
    int lo, hi;
    if constexpr (KIND == BATCH_AB) {
        lo = groups[combo * 2];
        hi = groups[combo * 2 + 2];
    } else {
        const int c = (KIND == BATCH_AA_EVEN) ? (int)(g & 1) : (int)((g & 1) ^ 1);
        lo = groups[combo * 2 + c];
        hi = groups[combo * 2 + c + 1];
    }
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int w = lo + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < hi; w += warps) {
        // item: (lattice, first row, segment, row groups)
        const int4 it = items[w];
        const BatchDesc<typename Storage<S>::C> &d = descs[it.x];
        if (g < d.g_base || g >= d.g_end) continue;  // warp-uniform
        const long long t = d.t_base + (g - d.g_base);
        T *base = static_cast<T *>(d.mem);
        const int rows = 32 >> d.lw;
        for (int q = 0; q < it.w; ++q) {
            const int y0 = it.y + q * rows;
            if constexpr (KIND == BATCH_AB) {
                const T *src = base + (size_t)(t & 1) * d.buf_elems;
                T *dst = base + (size_t)((t + 1) & 1) * d.buf_elems;
                item_ab<S, EQ, COLL, S == ST_F32, WALLS>(src, dst, d.nx, d.ny, d.pitch, d.plane, y0,
                                                   it.z, lane, d.lw, d.k, t, d.sr != 0);
            } else if constexpr (KIND == BATCH_AA_ODD) {
                item_aa_odd<S, EQ, COLL, S == ST_F32, WALLS>(base, d.nx, d.ny, d.pitch, d.plane, y0,
                                                       it.z, lane, d.lw, d.k, t, d.sr != 0);
            } else {
                item_aa_even<S, EQ, COLL, S == ST_F32, WALLS>(base, d.nx, d.ny, d.pitch, d.plane, y0,
                                                        it.z, lane, d.lw, d.k, t, d.sr != 0);
            }
        }
    }
}

template <int S> struct BatchLaunchT {
    template <int KIND, bool WALLS, int EQ, int COLL>
    static void launch_one(const BatchLaunch &a) {
        constexpr int bit = ((WALLS ? 1 : 0) * 3 + EQ) * 2 + COLL;
        if (!(a.combos & (1u << bit))) return;
        using D = BatchDesc<typename Storage<S>::C>;
        k_batch_step<S, KIND, EQ, COLL, WALLS><<<a.grid, a.block, 0, a.stream>>>(
            static_cast<const D *>(a.descs), a.items, a.groups, a.g, a.k);
    }
    template <int KIND, bool WALLS>
    static void launch_combos(const BatchLaunch &a) {
        launch_one<KIND, WALLS, EQ_GUIDED, COLL_OREG>(a);
        launch_one<KIND, WALLS, EQ_GUIDED, COLL_BGK>(a);
        launch_one<KIND, WALLS, EQ_POLY2, COLL_OREG>(a);
        launch_one<KIND, WALLS, EQ_POLY2, COLL_BGK>(a);
        launch_one<KIND, WALLS, EQ_GUIDED_LOCAL, COLL_OREG>(a);
        launch_one<KIND, WALLS, EQ_GUIDED_LOCAL, COLL_BGK>(a);
    }
    template <int KIND>
    static cudaError_t launch_kind(const BatchLaunch &a) {
        launch_combos<KIND, false>(a);
        launch_combos<KIND, true>(a);
        return cudaGetLastError();
    }
    static cudaError_t launch(const BatchLaunch &a) {
        if (a.layout == 0) return launch_kind<BATCH_AB>(a);
        cudaError_t e = launch_kind<BATCH_AA_EVEN>(a);
        if (e != cudaSuccess) return e;
        return launch_kind<BATCH_AA_ODD>(a);
    }
    static int occupancy(int layout, int block) {
        int n = 0;
        cudaError_t e = layout == 0
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                  &n, k_batch_step<S, BATCH_AB, EQ_GUIDED, COLL_OREG, false>, block, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                  &n, k_batch_step<S, BATCH_AA_ODD, EQ_GUIDED, COLL_OREG, false>, block, 0);
        return e == cudaSuccess ? n : 0;
    }
};

}  // namespace oreg

#define OREG_DEFINE_BATCH_LAUNCHERS(SUFFIX, S)                                          \
    namespace oreg {                                                                    \
    cudaError_t batch_step_##SUFFIX(const BatchLaunch &a) {                             \
        return BatchLaunchT<S>::launch(a);                                              \
    }                                                                                   \
    int batch_occupancy_##SUFFIX(int layout, int block) {                               \
        return BatchLaunchT<S>::occupancy(layout, block);                               \
    }                                                                                   \
    size_t batch_desc_size_##SUFFIX() { return sizeof(BatchDesc<typename Storage<S>::C>); } \
    }
