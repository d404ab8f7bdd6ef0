// Host-side launch interface between the C ABI (oreg_api.cu) and the kernels,
// which are instantiated once per storage format (oreg_st_*.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace oreg {

template <typename C> struct CollConst;

// Where a layout keeps the canonical state S_t (see canon_index).
enum { STATE_AB = 0, STATE_AA_EVEN = 1, STATE_AA_ODD = 2 };

// Geometry of a population state: planes of ny rows of `pitch` elements; the
// first nx elements of a row are nodes, the rest padding.
struct StateGeom {
    int nx, ny, pitch;
    size_t plane;  // elements per population plane
    int mode;      // STATE_*
};

struct StepArgs {
    void *src;         // A-B: buffer of S_t; AA: the single buffer
    void *dst;         // A-B: buffer of S_{t+1}; AA: unused
    int nx, ny, pitch;
    size_t plane;
    int passes;        // warp passes over a plane (warp_passes)
    int eq, coll, layout, parity;  // eq: kernel equilibrium kind (EQ_GUIDED_LOCAL for
                                   // the guided equilibrium at the local temperature)
    int comp;          // exact conserved-moment sums (FP32 only)
    int sr;            // stochastic rounding (half formats only)
    int walls;         // full-way bounce-back wall columns x = 0 and x = nx - 1
    long long t;       // time of the state being advanced
    int warps_per_block;
    const void *kconst;  // CollConst<C> of the storage's compute type
    cudaStream_t stream;
};

// Warp passes of the stream-collide kernels over a plane of ny rows of
// `pitch` elements (pitch a multiple of V): a pass covers 32 consecutive
// vectors of V elements in row-major order, rows back to back, so only the
// last pass of a lattice has idle lanes.  Every vector index of a plane fits
// an int (checked when a lattice is created).
inline long long warp_passes(int pitch, int ny, int V) {
    return ((long long)(pitch / V) * ny + 31) / 32;
}

enum { INIT_SHEAR = 0, INIT_SHOCK = 1, INIT_FIELDS = 2 };

struct InitSpec {
    int mode;
    double rho_a, rho_b;  // shear: rho0; shock: left/right density
    double u0, ex, ey;    // shear amplitude and direction e_perp
    int m, n;             // shear wave vector integers
    double ux_mean, uy_mean;  // shear: uniform mean flow
    int first_order;          // shear: add f^(1) of Eq. 5 from the analytic gradient
    double kx, ky;            // shear: wave vector 2 pi (m/nx, n/ny)
    double tau;               // relaxation time entering Eq. 5
    int x_split;          // shock split column
    const double *rho, *ux, *uy;  // fields mode: device arrays [rows][nx]
    int y0, rows;                 // rows initialised by this launch
};

struct ModeSpec {
    int active;
    int m, n;
    double ex, ey;
    const double *tab;  // [sin(2 pi m x/nx) | cos(..) over x, sin(2 pi n y/ny) | cos(..) over y]
};

#define OREG_DECLARE_LAUNCHERS(SUFFIX)                                                            \
    cudaError_t step_##SUFFIX(const StepArgs &a);                                                 \
    cudaError_t init_##SUFFIX(void *b, const StateGeom &g, const InitSpec &sp, int eq,            \
                              const CollConst<double> &kd, cudaStream_t s);                       \
    cudaError_t get_canonical_##SUFFIX(const void *b, const StateGeom &g, int x0, int y0, int wx, \
                                       int wy, const CollConst<double> &kd, double *out,          \
                                       cudaStream_t s);                                           \
    cudaError_t set_canonical_##SUFFIX(void *b, const StateGeom &g, int y0, int rows,             \
                                       const CollConst<double> &kd, const double *in,             \
                                       cudaStream_t s);                                           \
    cudaError_t moments_##SUFFIX(const void *b, const StateGeom &g, int y0, int rows,             \
                                 const CollConst<double> &kd, double *r, double *ux, double *uy,  \
                                 double *th, cudaStream_t s);                                     \
    cudaError_t reduce_##SUFFIX(const void *b, const StateGeom &g, const CollConst<double> &kd,   \
                                const ModeSpec &m, double *partials, int nblocks, double *out,    \
                                cudaStream_t s);

OREG_DECLARE_LAUNCHERS(f64)
OREG_DECLARE_LAUNCHERS(f32)
OREG_DECLARE_LAUNCHERS(f16)
OREG_DECLARE_LAUNCHERS(bf16)
// Stream-collide only, FP32 storage with the FP64 collision (ST_F32_C64); the
// state is that of FP32 storage, so initialisation, readback and reductions
// use the f32 launchers.
cudaError_t step_f32c64(const StepArgs &a);

// One launch of the batched stream-collide kernel (see oreg_batch_kernels.cuh).
// Default warp passes (32 consecutive vectors each) per batched work item: a
// warp takes up to this many consecutive passes over one lattice, reading the
// lattice's descriptor once (olb_batch_params.item_passes overrides it).
constexpr int BATCH_ITEM_PASSES = 4;

// One slot of a batch: a (walls, equilibrium kind, collision) kernel and the
// collision constants of one class of lattices (all but 1 - 1/tau).
struct BatchSlot {
    int combo;            // (walls * 3 + eq) * 2 + coll
    const void *kconst;   // host CollConst<C> of the class (copied into the launch)
};

struct BatchLaunch {
    const void *descs;        // BatchDesc<C>[]
    const int4 *items;        // work items (descriptor, first vector, 0, passes), grouped
    const int *groups;        // device: item offsets of the (slot, parity) groups
    const long long *g;       // device: global step counter of this round
    int k;                    // step within the round
    int layout;
    int first_slot, nslots;   // slots to launch (first_slot .. first_slot + nslots - 1),
                              // one kernel each per step
    const BatchSlot *slots;   // every slot of the batch (indexed by slot)
    int grid, block;
    cudaStream_t stream;
};

#define OREG_DECLARE_BATCH_LAUNCHERS(SUFFIX)                 \
    cudaError_t batch_step_##SUFFIX(const BatchLaunch &a);   \
    int batch_occupancy_##SUFFIX(int layout, int block);     \
    size_t batch_desc_size_##SUFFIX();                       \
    size_t batch_const_size_##SUFFIX();

OREG_DECLARE_BATCH_LAUNCHERS(f64)
OREG_DECLARE_BATCH_LAUNCHERS(f32)
OREG_DECLARE_BATCH_LAUNCHERS(f16)
OREG_DECLARE_BATCH_LAUNCHERS(bf16)

constexpr int RED_BLOCKS_MAX = 1216;  // fixed reduction grid (8 x 152 SMs)
constexpr int RED_QUANTITIES = 6;

}  // namespace oreg
