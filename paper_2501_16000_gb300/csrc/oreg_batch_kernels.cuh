// Batched stream-collide: one kernel advances many independent lattices of
// any size by one time step, its warps striding over a flattened table of
// warp work items (runs of warp passes over one lattice's planes).  The
// grid is either resident as a whole (persistent) or oversubscribed, so that
// blocks start as earlier ones finish.
//
// Every lattice keeps its own population memory, geometry and relaxation
// time in a device descriptor; the rest of its collision constants belong to
// its slot (below).  A device-resident global step counter g decides, per
// lattice, whether it is active in this launch (g_base <= g < g_end) and at
// which local time t = t_base + (g - g_base), which selects the A-B buffer or
// the AA parity.  The launches of K steps and one counter increment are
// captured in a CUDA graph; joining and leaving lattices only rewrite the
// descriptor, item and group tables (stream-ordered copies), and the graph is
// captured again only when a lattice brings a new slot.
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
    size_t plane;         // elements per plane
    size_t buf_elems;     // elements per population buffer
    long long t_base;     // lattice time when the global step counter was g_base
    long long g_base;     // first global step the lattice takes part in
    long long g_end;      // first global step it no longer takes part in
    int sr;               // stochastic rounding of half formats
    C lam;                // 1 - 1/tau of this lattice (the collision constants
                          // but lam come from its constant class)
};

// Lattices are grouped into slots: one (walls, equilibrium kind, collision)
// kernel and one constant class, i.e. the same collision constants apart from
// 1 - 1/tau (same theta, rho0 and equilibrium).  The class constants reach
// the kernel as a launch parameter, like the single-lattice kernels' (the
// compiler re-reads them from the parameter bank instead of holding them in
// registers), and each lattice's lam comes from its descriptor.  Work items
// are grouped by (slot, parity class): group = slot * 2 + c, with
// c = (t_base - g_base) & 1 the lattice's fixed offset between its own time
// and the global step, so that at global step g every lattice of class c has
// time parity (g + c) & 1.  groups[0 .. 2 * slots] are the item offsets of
// the groups; one launch per slot and step (per parity kernel for the in-place
// layout) walks its items.
enum { BATCH_AB = 0, BATCH_AA_EVEN = 1, BATCH_AA_ODD = 2 };

// At most 128 threads x 4 blocks per SM (a 128-register cap, 16 warps): with
// the class constants in the parameter bank the half-format kernels fit in
// 128 registers without spilling (158 when the constants came from the
// descriptor in global memory, 12 warps).
constexpr int BATCH_MAX_THREADS = 128;
constexpr int BATCH_MIN_BLOCKS = 4;
template <int S, int KIND, int EQ, int COLL, bool WALLS>
__global__ void __launch_bounds__(BATCH_MAX_THREADS, BATCH_MIN_BLOCKS)
    k_batch_step(const BatchDesc<typename Storage<S>::C> *__restrict__ descs,
                 const int4 *__restrict__ items, const int *__restrict__ groups,
                 const long long *__restrict__ g_round, int k, int slot,
                 const CollConst<typename Storage<S>::C> kc) {
    using T = typename Storage<S>::T;
    const long long g = *g_round + k;
    int lo, hi;
    if constexpr (KIND == BATCH_AB) {
        lo = groups[slot * 2];
        hi = groups[slot * 2 + 2];
    } else {
        const int c = (KIND == BATCH_AA_EVEN) ? (int)(g & 1) : (int)((g & 1) ^ 1);
        lo = groups[slot * 2 + c];
        hi = groups[slot * 2 + c + 1];
    }
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int w = lo + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < hi; w += warps) {
        // item: (lattice, first vector, 0, warp passes)
        const int4 it = items[w];
        const BatchDesc<typename Storage<S>::C> &d = descs[it.x];
        if (g < d.g_base || g >= d.g_end) continue;  // warp-uniform
        const long long t = d.t_base + (g - d.g_base);
        T *base = static_cast<T *>(d.mem);
        CollConst<typename Storage<S>::C> kk = kc;
        kk.lam = d.lam;
        for (int q = 0; q < it.w; ++q) {
            const int v0 = it.y + q * 32;
            if constexpr (KIND == BATCH_AB) {
                const T *src = base + (size_t)(t & 1) * d.buf_elems;
                T *dst = base + (size_t)((t + 1) & 1) * d.buf_elems;
                item_ab<S, EQ, COLL, S == ST_F32, WALLS>(src, dst, d.nx, d.ny, d.pitch, d.plane, v0,
                                                         lane, kk, t, d.sr != 0);
            } else if constexpr (KIND == BATCH_AA_ODD) {
                item_aa_odd<S, EQ, COLL, S == ST_F32, WALLS>(base, d.nx, d.ny, d.pitch, d.plane, v0,
                                                             lane, kk, t, d.sr != 0);
            } else {
                item_aa_even<S, EQ, COLL, S == ST_F32, WALLS>(base, d.nx, d.ny, d.pitch, d.plane,
                                                              v0, lane, kk, t, d.sr != 0);
            }
        }
    }
}

template <int S> struct BatchLaunchT {
    using C = typename Storage<S>::C;
    using D = BatchDesc<C>;
    template <int KIND, bool WALLS, int EQ, int COLL>
    static void launch_one(const BatchLaunch &a, int s) {
        const CollConst<C> &kc = *static_cast<const CollConst<C> *>(a.slots[s].kconst);
        k_batch_step<S, KIND, EQ, COLL, WALLS><<<a.grid, a.block, 0, a.stream>>>(
            static_cast<const D *>(a.descs), a.items, a.groups, a.g, a.k, s, kc);
    }
    template <int KIND, bool WALLS, int EQ>
    static void launch_coll(const BatchLaunch &a, int s, int coll) {
        if (coll == COLL_OREG) launch_one<KIND, WALLS, EQ, COLL_OREG>(a, s);
        else launch_one<KIND, WALLS, EQ, COLL_BGK>(a, s);
    }
    template <int KIND, bool WALLS>
    static void launch_eq(const BatchLaunch &a, int s, int eq, int coll) {
        if (eq == EQ_GUIDED) launch_coll<KIND, WALLS, EQ_GUIDED>(a, s, coll);
        else if (eq == EQ_POLY2) launch_coll<KIND, WALLS, EQ_POLY2>(a, s, coll);
        else launch_coll<KIND, WALLS, EQ_GUIDED_LOCAL>(a, s, coll);
    }
    // combo = (walls * 3 + eq) * 2 + coll
    template <int KIND>
    static cudaError_t launch_kind(const BatchLaunch &a) {
        for (int s = a.first_slot; s < a.first_slot + a.nslots; ++s) {
            const int combo = a.slots[s].combo;
            const int coll = combo & 1, eq = (combo >> 1) % 3, walls = combo / 6;
            if (walls) launch_eq<KIND, true>(a, s, eq, coll);
            else launch_eq<KIND, false>(a, s, eq, coll);
        }
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
    size_t batch_const_size_##SUFFIX() { return sizeof(CollConst<typename Storage<S>::C>); } \
    }
