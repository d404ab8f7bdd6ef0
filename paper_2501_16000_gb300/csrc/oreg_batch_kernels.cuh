// Batched stream-collide: one persistent kernel advances many independent
// lattices of any size by one time step, walking a flattened table of warp
// work items (one row segment of one lattice each).
//
// Every lattice keeps its own population memory, geometry, relaxation time
// and equilibrium constants in a device descriptor.  A device-resident global
// step counter g decides, per lattice, whether it is active in this launch
// (g_base <= g < g_end) and at which local time t = t_base + (g - g_base),
// which selects the A-B buffer or the AA parity.  K launches and one counter
// increment are captured once in a CUDA graph; joining and leaving lattices
// only rewrite the descriptor and item tables, so the graph is never
// re-captured.
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
    CollConst<C> k;
};

// One work item: x = descriptor index, y = row, z = row segment.
template <int S, int LAYOUT, int EQ, int COLL>
__device__ __forceinline__ void batch_item(const BatchDesc<typename Storage<S>::C> &d, long long t,
                                           int y, int seg, int lane) {
    using T = typename Storage<S>::T;
    T *base = static_cast<T *>(d.mem);
    if constexpr (LAYOUT == 0) {
        const T *src = base + (size_t)(t & 1) * d.buf_elems;
        T *dst = base + (size_t)((t + 1) & 1) * d.buf_elems;
        item_ab<S, EQ, COLL, false>(src, dst, d.nx, d.ny, d.pitch, d.plane, y, seg, lane, d.k, t,
                                    d.sr != 0);
    } else if (t & 1) {
        item_aa_odd<S, EQ, COLL, false>(base, d.nx, d.ny, d.pitch, d.plane, y, seg, lane, d.k, t,
                                        d.sr != 0);
    } else {
        item_aa_even<S, EQ, COLL, false>(base, d.nx, d.pitch, d.plane, y, seg, lane, d.k, t,
                                         d.sr != 0);
    }
}

template <int S, int LAYOUT>
__global__ void __launch_bounds__(256)
    k_batch_step(const BatchDesc<typename Storage<S>::C> *__restrict__ descs,
                 const int4 *__restrict__ items, const int *__restrict__ n_items,
                 const long long *__restrict__ g_round, int k) {
    const long long g = *g_round + k;
    const int n = *n_items;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n; w += warps) {
        const int4 it = items[w];
        const BatchDesc<typename Storage<S>::C> &d = descs[it.x];
        if (g < d.g_base || g >= d.g_end) continue;  // warp-uniform
        const long long t = d.t_base + (g - d.g_base);
        const int sel = d.eq * 2 + d.coll;
        if (sel == 0) batch_item<S, LAYOUT, EQ_GUIDED, COLL_OREG>(d, t, it.y, it.z, lane);
        else if (sel == 1) batch_item<S, LAYOUT, EQ_GUIDED, COLL_BGK>(d, t, it.y, it.z, lane);
        else if (sel == 2) batch_item<S, LAYOUT, EQ_POLY2, COLL_OREG>(d, t, it.y, it.z, lane);
        else batch_item<S, LAYOUT, EQ_POLY2, COLL_BGK>(d, t, it.y, it.z, lane);
    }
}

template <int S> struct BatchLaunchT {
    static cudaError_t launch(const BatchLaunch &a) {
        using D = BatchDesc<typename Storage<S>::C>;
        const D *descs = static_cast<const D *>(a.descs);
        if (a.layout == 0)
            k_batch_step<S, 0><<<a.grid, a.block, 0, a.stream>>>(descs, a.items, a.n_items, a.g, a.k);
        else
            k_batch_step<S, 1><<<a.grid, a.block, 0, a.stream>>>(descs, a.items, a.n_items, a.g, a.k);
        return cudaGetLastError();
    }
    static int occupancy(int layout, int block) {
        int n = 0;
        cudaError_t e = layout == 0
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_step<S, 0>, block, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_step<S, 1>, block, 0);
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
