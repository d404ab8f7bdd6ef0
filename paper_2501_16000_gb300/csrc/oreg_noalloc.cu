// olb_diagnostics_noalloc: the FP64 diagnostics reduction over a population
// state held in caller memory, without allocating any memory.
//
// Who needs this: callers that own the device memory budget themselves and
// cannot let the library call cudaMalloc, e.g. a serving loop that admits
// work against a fixed HBM budget it accounts byte by byte, or a host loop on
// a latency budget where cudaMalloc/cudaFree would add an implicit device
// synchronisation.  They can keep populations in their own buffers (laid out
// as liboreg lays out a lattice) and still read the mass, momentum and
// non-finite count.
//
// The reduction partials live in a file-scope __device__ array of fixed size
// instead of library-allocated scratch.  Every GPU that loads the library
// holds that array until the process exits.  All calls share it, so calls
// whose work overlaps on the GPU (for example on two streams) race.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "oreg.h"
#include "oreg_aux.cuh"
#include "oreg_consts.h"

namespace oreg {
void set_last_error_message(const char *msg);
}

namespace {

using namespace oreg;

constexpr int NOALLOC_MAX_ROWS = 16384;  // == OLB_NOALLOC_MAX_ROWS in oreg.h
constexpr int NOALLOC_Q = 4;             // mass, momentum x, momentum y, non-finite count
constexpr int NOALLOC_THREADS = 256;
constexpr int MAX_DEVICES = 64;

static_assert(NOALLOC_MAX_ROWS == OLB_NOALLOC_MAX_ROWS, "header and implementation disagree");

// One partial per lattice row; 16384 x 4 doubles = 512 KiB per device.
static __device__ __align__(256) double g_row_partials[NOALLOC_MAX_ROWS * NOALLOC_Q];

// Device address of g_row_partials per device, looked up once per device.
double *g_partials_addr[MAX_DEVICES];
std::mutex g_partials_mu;

olb_status noalloc_fail(olb_status st, const char *msg) {
    set_last_error_message(msg);
    return st;
}

// Row y of the lattice: sums of rho, j_x, j_y over finite nodes and the
// number of nodes with a non-finite population, into partials[y].
template <int S>
__global__ void __launch_bounds__(NOALLOC_THREADS)
    k_row_sums(const typename Storage<S>::T *base, StateGeom g, const CollConst<double> kd,
               double *partials) {
    const int y = blockIdx.x;
    double acc[NOALLOC_Q] = {0, 0, 0, 0};
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
        double f[9];
        canon_node<S>(base, x, y, g, kd.shift, f);
        double r = 0, jx = 0, jy = 0;
        bool finite = true;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            finite = finite && isfinite(f[i]);
            r += f[i];
            jx += cx_of(i) * f[i];
            jy += cy_of(i) * f[i];
        }
        if (!finite) {
            acc[3] += 1.0;
            continue;
        }
        acc[0] += r;
        acc[1] += jx;
        acc[2] += jy;
    }
    __shared__ double sh[NOALLOC_THREADS / 32][NOALLOC_Q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NOALLOC_Q; ++q) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) sh[warp][q] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NOALLOC_Q; ++q) {
            double v = lane < NOALLOC_THREADS / 32 ? sh[lane][q] : 0.0;
            v = warp_sum(v);
            if (lane == 0) partials[(size_t)y * NOALLOC_Q + q] = v;
        }
    }
}

// Sum of the ny row partials (every one was written by k_row_sums of the
// same call, so nothing needs clearing) into out[0..3].
__global__ void __launch_bounds__(NOALLOC_THREADS)
    k_rows_final(const double *partials, int rows, double *out) {
    double acc[NOALLOC_Q] = {0, 0, 0, 0};
    for (int r = threadIdx.x; r < rows; r += blockDim.x)
#pragma unroll
        for (int q = 0; q < NOALLOC_Q; ++q) acc[q] += partials[(size_t)r * NOALLOC_Q + q];
    __shared__ double sh[NOALLOC_THREADS / 32][NOALLOC_Q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NOALLOC_Q; ++q) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) sh[warp][q] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NOALLOC_Q; ++q) {
            double v = lane < NOALLOC_THREADS / 32 ? sh[lane][q] : 0.0;
            v = warp_sum(v);
            if (lane == 0) out[q] = v;
        }
    }
}

template <int S>
cudaError_t launch_rows(const void *base, const StateGeom &g, const CollConst<double> &kd,
                        double *partials, double *out, cudaStream_t s) {
    k_row_sums<S><<<g.ny, NOALLOC_THREADS, 0, s>>>(
        static_cast<const typename Storage<S>::T *>(base), g, kd, partials);
    k_rows_final<<<1, NOALLOC_THREADS, 0, s>>>(partials, g.ny, out);
    return cudaGetLastError();
}

}  // namespace

extern "C" olb_status olb_diagnostics_noalloc(const void *d_populations, const olb_params *p,
                                              int64_t t, double *d_out) {
    char msg[256];
    if (!d_populations || !p || !d_out)
        return noalloc_fail(OLB_ERR_INVALID, "d_populations, p and d_out must not be NULL");
    if (p->nx < 1 || p->ny < 1)
        return noalloc_fail(OLB_ERR_INVALID, "nx, ny must be >= 1");
    if (p->ny > NOALLOC_MAX_ROWS) {
        snprintf(msg, sizeof msg,
                 "olb_diagnostics_noalloc handles at most %d rows (its fixed scratch holds one "
                 "partial per row); got ny = %d",
                 NOALLOC_MAX_ROWS, p->ny);
        return noalloc_fail(OLB_ERR_INVALID, msg);
    }
    if (t < 0) return noalloc_fail(OLB_ERR_INVALID, "t must be >= 0");
    if (p->storage < OLB_F64 || p->storage > OLB_BF16_SHIFTED)
        return noalloc_fail(OLB_ERR_INVALID, "unknown storage");
    if (p->layout != OLB_LAYOUT_AB && p->layout != OLB_LAYOUT_AA)
        return noalloc_fail(OLB_ERR_INVALID, "unknown layout");
    if (p->eq != OLB_EQ_GUIDED && p->eq != OLB_EQ_POLY2)
        return noalloc_fail(OLB_ERR_INVALID, "unknown equilibrium");
    if (!(std::isfinite(p->rho0) && p->rho0 > 0) || !(std::isfinite(p->tau) && p->tau > 0.5) ||
        (p->eq == OLB_EQ_GUIDED && !(p->theta > 0 && p->theta < 1)))
        return noalloc_fail(OLB_ERR_INVALID, "rho0, tau or theta out of range");
    if (reinterpret_cast<uintptr_t>(d_populations) % 16 != 0)
        return noalloc_fail(OLB_ERR_INVALID, "d_populations must be 16-byte aligned");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "cudaGetDevice: %s", cudaGetErrorString(e));
        return noalloc_fail(OLB_ERR_CUDA, msg);
    }
    if (dev < 0 || dev >= MAX_DEVICES) return noalloc_fail(OLB_ERR_INVALID, "device index out of range");
    double *partials = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_partials_mu);
        if (!g_partials_addr[dev]) {
            // first call on this device (which is current): device address of the array
            void *addr = nullptr;
            e = cudaGetSymbolAddress(&addr, g_row_partials);
            if (e != cudaSuccess) {
                snprintf(msg, sizeof msg, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
                return noalloc_fail(OLB_ERR_CUDA, msg);
            }
            g_partials_addr[dev] = static_cast<double *>(addr);
        }
        partials = g_partials_addr[dev];
    }

    const int esize = p->storage == OLB_F64 ? 8 : (p->storage == OLB_F32 ? 4 : 2);
    const int V = 16 / esize;
    StateGeom g;
    g.nx = p->nx;
    g.ny = p->ny;
    g.pitch = ((p->nx + V - 1) / V) * V;
    g.plane = (size_t)g.pitch * p->ny;
    const char *base = static_cast<const char *>(d_populations);
    if (p->layout == OLB_LAYOUT_AB) {
        g.mode = STATE_AB;
        base += (size_t)(t & 1) * 9 * g.plane * esize;
    } else {
        g.mode = (t & 1) ? STATE_AA_ODD : STATE_AA_EVEN;
    }
    // the FP64 constants liboreg uses for a lattice with these parameters
    // (shifts exactly those of the stored format)
    const CollConst<double> kd = make_const_f64_for(p);
    cudaStream_t s = static_cast<cudaStream_t>(p->cuda_stream);
    switch (p->storage) {
        case OLB_F64: e = launch_rows<ST_F64>(base, g, kd, partials, d_out, s); break;
        case OLB_F32: e = launch_rows<ST_F32>(base, g, kd, partials, d_out, s); break;
        case OLB_F16_SHIFTED: e = launch_rows<ST_F16>(base, g, kd, partials, d_out, s); break;
        default: e = launch_rows<ST_BF16>(base, g, kd, partials, d_out, s); break;
    }
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "launching the no-allocation reduction: %s", cudaGetErrorString(e));
        return noalloc_fail(OLB_ERR_CUDA, msg);
    }
    return OLB_OK;
}
