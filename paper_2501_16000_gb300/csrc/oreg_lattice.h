// Internal definition of the opaque olb_lattice handle (shared by the C-ABI
// translation units; not part of the public header).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

#include "oreg.h"
#include "oreg_device.cuh"
#include "oreg_launch.h"

struct olb_batch;

struct olb_lattice {
    olb_params p;
    int V;
    size_t esize;
    int pitch;
    size_t plane;         // elements per plane
    size_t buf_elems;     // elements per population buffer (9 planes)
    int nbuf;
    void *mem;            // population memory (2 buffers for A-B, 1 for AA)
    bool own_mem;
    cudaStream_t stream;        // stream of every call on the lattice (olb_set_stream)
    cudaStream_t owned_stream;  // stream the library created for it, or NULL
    int64_t t;            // time of the canonical state; -1 = uninitialised
    int comp;
    int sr;               // stochastic rounding of half formats
    int f64_coll;         // FP32 storage: collision in FP64 (OLB_OPT_F64_COLLISION)
    int warps_per_block;
    int num_sms;
    double *d_red;        // reduction partials + result (library scratch, lazy)
    double *h_red;        // pinned host copy of the result (lazy)
    int red_blocks;
    void *d_chunk;        // readback scratch (lazy)
    size_t chunk_bytes;
    // Field upload and moments readback alternate between two halves of the
    // scratch and run their copies on copy_stream, so that the copies of one
    // chunk overlap the conversion kernel of the other (lazy).
    cudaStream_t copy_stream;
    cudaEvent_t ev_main[2];  // recorded on the lattice's stream, per half
    cudaEvent_t ev_copy[2];  // recorded on copy_stream, per half
    double *d_tab;        // shear-mode sin/cos tables (lazy), for (tab_m, tab_n)
    double *h_tab;
    int tab_m, tab_n;
    oreg::CollConst<double> kd;     // FP64 constants (shift as stored type's shift)
    oreg::CollConst<float> kf;      // FP32 constants (F32, F16, BF16 compute)
    olb_batch *batch;               // batch the lattice currently belongs to, or NULL
    unsigned long long *d_cmp;      // olb_compare result scratch (lazy)
};

namespace oreg {
// Records the message of a failed call for olb_last_error() (oreg_api.cu).
void set_last_error_message(const char *msg);

// NVTX range over one C-ABI call (visible in Nsight timelines; a no-op when
// no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Equilibrium kind of the stream-collide kernels for a lattice.
inline int kernel_eq(const olb_params *p) {
    if (p->eq == OLB_EQ_GUIDED && p->theta_mode == OLB_THETA_LOCAL) return EQ_GUIDED_LOCAL;
    return p->eq == OLB_EQ_GUIDED ? EQ_GUIDED : EQ_POLY2;
}

// Geometry of the lattice's canonical state at its current time.
inline StateGeom geom(const olb_lattice *L) {
    StateGeom g;
    g.nx = L->p.nx;
    g.ny = L->p.ny;
    g.pitch = L->pitch;
    g.plane = L->plane;
    g.mode = L->p.layout == OLB_LAYOUT_AB ? STATE_AB : ((L->t & 1) ? STATE_AA_ODD : STATE_AA_EVEN);
    return g;
}

// Buffer holding S_t.
inline void *state_base(const olb_lattice *L) {
    const size_t bytes = L->buf_elems * L->esize;
    if (L->p.layout == OLB_LAYOUT_AA) return L->mem;
    return static_cast<char *>(L->mem) + (size_t)(L->t & 1) * bytes;
}
}  // namespace oreg
